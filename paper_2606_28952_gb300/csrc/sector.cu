// sector.cu -- spin-resolved product sectors (Sec. 2.4, eq. fcidim) and their
// rank / unrank maps.
//
// A configuration b splits into a low half b_lo (n_lo qubits; the alpha
// string of a molecule) and a high half b_hi (the beta string).  Inside block
// r = (k_lo, k_hi) its index is off_r + rank(b_hi) * D_lo^r + rank(b_lo),
// where rank is the colex rank among strings with the same popcount,
//   rank(b) = sum_j C(p_j, j + 1),  p_0 < p_1 < ... the set-bit positions,
// which equals the position of b in the ascending list of such strings.  The
// binomial table below is that ranking's only constant; the apply kernels read
// per-half lookup tables that k_rank_table fills with the same function.
#include <algorithm>
#include <vector>

#include "ps_internal.cuh"

namespace ps {
namespace {

__constant__ uint64_t c_binom[33][33];  // C(p, j) for 0 <= p, j <= 32
constexpr int kBinomDevices = 64;
bool g_binom_ready[kBinomDevices] = {};  // constant memory is per device

void ensure_binom() {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < kBinomDevices && g_binom_ready[dev]) return;
    uint64_t b[33][33] = {};
    for (int p = 0; p <= 32; ++p) {
        b[p][0] = 1;
        for (int j = 1; j <= p; ++j) b[p][j] = b[p - 1][j - 1] + (j <= p - 1 ? b[p - 1][j] : 0);
    }
    PS_CUDA(cudaMemcpyToSymbol(c_binom, b, sizeof(b)));
    if (dev >= 0 && dev < kBinomDevices) g_binom_ready[dev] = true;
}

__device__ __forceinline__ uint64_t colex_rank(uint32_t s) {
    uint64_t r = 0;
    int j = 0;
    while (s) {
        int p = __ffs(s) - 1;
        r += c_binom[p][j + 1];
        ++j;
        s &= s - 1;
    }
    return r;
}

// k-subset of {0..bits-1} with colex rank r (r < C(bits, k))
__device__ __forceinline__ uint32_t colex_unrank(int bits, int k, uint64_t r) {
    uint32_t s = 0;
    int p = bits - 1;
    for (int j = k; j >= 1; --j) {
        while (p >= 0 && c_binom[p][j] > r) --p;
        s |= 1u << p;
        r -= c_binom[p][j];
        --p;
    }
    return s;
}

__global__ void k_rank_table(int bits, uint32_t *rank) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1ll << bits)) return;
    rank[s] = (uint32_t)colex_rank((uint32_t)s);
}

__global__ void k_list_table(int bits, const uint32_t *rank, const int64_t *off_by_pop,
                             uint32_t *list) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1ll << bits)) return;
    list[off_by_pop[__popc((uint32_t)s)] + rank[s]] = (uint32_t)s;
}

__global__ void k_sector_rank(SectorView v, const uint64_t *cfg, int64_t n, int64_t *idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t b = cfg[i];
    if (v.kind == PAULI_SECTOR_FULL) {
        idx[i] = (v.n < 64 && (b >> v.n) != 0) ? -1 : (int64_t)b;
        return;
    }
    if ((b >> v.n) != 0) { idx[i] = -1; return; }
    uint32_t lo = (uint32_t)(b & ((1ull << v.n_lo) - 1ull));
    uint32_t hi = (uint32_t)(b >> v.n_lo);
    int blk = v.blk_of_khi[cls_hi(v, hi)];
    if (blk < 0 || cls_lo(v, lo) != v.klo[blk]) { idx[i] = -1; return; }
    if (v.irr) {
        // ranks inside (popcount, irrep) classes come from the tables
        idx[i] = v.off[blk] + (int64_t)v.rank_hi[hi] * v.dlo[blk] + (int64_t)v.rank_lo[lo];
        return;
    }
    idx[i] = v.off[blk] + (int64_t)colex_rank(hi) * v.dlo[blk] + (int64_t)colex_rank(lo);
}

__global__ void k_sector_unrank(SectorView v, const int64_t *idx, int64_t n, uint64_t *cfg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t k = idx[i];
    if (k < 0 || k >= v.dim) { cfg[i] = ~0ull; return; }
    if (v.kind == PAULI_SECTOR_FULL) { cfg[i] = (uint64_t)k; return; }
    int blk = 0;
    while (blk + 1 < v.nblk && v.off[blk + 1] <= k) ++blk;
    int64_t rem = k - v.off[blk];
    uint64_t rhi = (uint64_t)(rem / v.dlo[blk]);
    uint64_t rlo = (uint64_t)(rem % v.dlo[blk]);
    uint32_t hi, lo;
    if (v.irr) {
        hi = v.list_hi[v.lst_hi_off[blk] + rhi];
        lo = v.list_lo[v.lst_lo_off[blk] + rlo];
    } else {
        hi = colex_unrank(v.n_hi, v.khi[blk], rhi);
        lo = colex_unrank(v.n_lo, v.klo[blk], rlo);
    }
    cfg[i] = (uint64_t)lo | ((uint64_t)hi << v.n_lo);
}

inline uint64_t binom_host(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int j = 1; j <= k; ++j) r = r * (uint64_t)(n - k + j) / (uint64_t)j;
    return r;
}

}  // namespace

void build_sector_tables(pauli_sector *s, cudaStream_t st) {
    ensure_binom();
    SectorView &v = s->v;
    if (v.kind == PAULI_SECTOR_FULL) {
        v.rank_lo = v.rank_hi = v.list_lo = v.list_hi = nullptr;
        return;
    }
    const int64_t nlo = 1ll << v.n_lo, nhi = 1ll << v.n_hi;
    const int64_t total = 2 * (nlo + nhi);
    s->tables = static_cast<uint32_t *>(dev_alloc(s->al, total * sizeof(uint32_t)));
    uint32_t *rank_lo = s->tables, *list_lo = rank_lo + nlo;
    uint32_t *rank_hi = list_lo + nlo, *list_hi = rank_hi + nhi;
    if (v.irr) {
        // (popcount, irrep) classes: ranks and lists by counting on the host
        for (int half = 0; half < 2; ++half) {
            const int bits = half ? v.n_hi : v.n_lo;
            const uint32_t *m = half ? v.irr_hi : v.irr_lo;
            std::vector<int64_t> off(kMaxCls + 1, 0);
            const int64_t cnt = 1ll << bits;
            std::vector<uint32_t> rk(cnt), ls(cnt);
            std::vector<int64_t> count(kMaxCls + 1, 0);
            for (int64_t t = 0; t < cnt; ++t) rk[t] = (uint32_t)count[half_cls((uint32_t)t, 1, m)]++;
            off[0] = 0;
            for (int c = 0; c < kMaxCls; ++c) off[c + 1] = off[c] + count[c];
            for (int64_t t = 0; t < cnt; ++t) ls[off[half_cls((uint32_t)t, 1, m)] + rk[t]] = (uint32_t)t;
            PS_CUDA(cudaMemcpyAsync(half ? rank_hi : rank_lo, rk.data(), cnt * 4, cudaMemcpyHostToDevice, st));
            PS_CUDA(cudaMemcpyAsync(half ? list_hi : list_lo, ls.data(), cnt * 4, cudaMemcpyHostToDevice, st));
            PS_CUDA(cudaStreamSynchronize(st));
            for (int r = 0; r < v.nblk; ++r) (half ? v.lst_hi_off : v.lst_lo_off)[r] = off[half ? v.khi[r] : v.klo[r]];
        }
        v.rank_lo = rank_lo;
        v.list_lo = list_lo;
        v.rank_hi = rank_hi;
        v.list_hi = list_hi;
        return;
    }
    for (int half = 0; half < 2; ++half) {
        const int bits = half ? v.n_hi : v.n_lo;
        std::vector<int64_t> off(bits + 2, 0);
        for (int k = 0; k <= bits; ++k) off[k + 1] = off[k] + (int64_t)binom_host(bits, k);
        for (int r = 0; r < v.nblk; ++r) (half ? v.lst_hi_off : v.lst_lo_off)[r] = off[half ? v.khi[r] : v.klo[r]];
        DevBuf<int64_t> d_off(s->al, bits + 2);
        PS_CUDA(cudaMemcpyAsync(d_off.p, off.data(), (bits + 2) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        uint32_t *rk = half ? rank_hi : rank_lo;
        uint32_t *ls = half ? list_hi : list_lo;
        const int64_t cnt = 1ll << bits;
        k_rank_table<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(bits, rk);
        PS_LAUNCH_CHECK();
        k_list_table<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(bits, rk, d_off.p, ls);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaStreamSynchronize(st));
    }
    v.rank_lo = rank_lo;
    v.list_lo = list_lo;
    v.rank_hi = rank_hi;
    v.list_hi = list_hi;
}

void sector_rank(const SectorView &v, const uint64_t *cfg, int64_t n, int64_t *idx, cudaStream_t st) {
    ensure_binom();
    if (n <= 0) return;
    k_sector_rank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, cfg, n, idx);
    PS_LAUNCH_CHECK();
}

void sector_unrank(const SectorView &v, const int64_t *idx, int64_t n, uint64_t *cfg,
                   cudaStream_t st) {
    ensure_binom();
    if (n <= 0) return;
    k_sector_unrank<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, idx, n, cfg);
    PS_LAUNCH_CHECK();
}

// host-side geometry of a sector (dimensions, offsets, block lookup).  With
// qubit_irrep (n labels 0..7; point-group blocks) klo / khi are the classes
// popcount * 8 + irrep of each block's halves, else popcounts.
void init_sector_view(SectorView &v, int n, int kind, int n_lo, int nb, const int *klo, const int *khi,
                      const int *qubit_irrep) {
    v = SectorView();
    v.n = n;
    v.kind = kind;
    for (int i = 0; i < kMaxCls; ++i) v.blk_of_khi[i] = -1;
    if (kind == PAULI_SECTOR_FULL) {
        v.n_lo = n_lo;
        v.n_hi = n - n_lo;
        v.nblk = 1;
        v.klo[0] = -1;
        v.khi[0] = -1;
        v.off[0] = 0;
        v.dlo[0] = 1ll << v.n_lo;
        v.dhi[0] = 1ll << v.n_hi;
        v.off[1] = v.dim = 1ll << n;
        v.row_off[0] = 0;
        v.row_off[1] = v.nrows = v.dhi[0];
        return;
    }
    v.n_lo = n_lo;
    v.n_hi = n - n_lo;
    v.nblk = nb;
    std::vector<int64_t> cnt_lo, cnt_hi;
    if (qubit_irrep) {
        v.irr = 1;
        for (int j = 0; j < 3; ++j) {
            v.irr_lo[j] = v.irr_hi[j] = 0u;
            for (int q = 0; q < v.n_lo; ++q)
                if ((qubit_irrep[q] >> j) & 1) v.irr_lo[j] |= 1u << q;
            for (int q = 0; q < v.n_hi; ++q)
                if ((qubit_irrep[v.n_lo + q] >> j) & 1) v.irr_hi[j] |= 1u << q;
        }
        cnt_lo.assign(kMaxCls, 0);
        cnt_hi.assign(kMaxCls, 0);
        for (int64_t t = 0; t < (1ll << v.n_lo); ++t) ++cnt_lo[half_cls((uint32_t)t, 1, v.irr_lo)];
        for (int64_t t = 0; t < (1ll << v.n_hi); ++t) ++cnt_hi[half_cls((uint32_t)t, 1, v.irr_hi)];
    }
    int64_t off = 0, row = 0;
    for (int r = 0; r < nb; ++r) {
        v.klo[r] = klo[r];
        v.khi[r] = khi[r];
        v.dlo[r] = v.irr ? cnt_lo[klo[r]] : (int64_t)binom_host(v.n_lo, klo[r]);
        v.dhi[r] = v.irr ? cnt_hi[khi[r]] : (int64_t)binom_host(v.n_hi, khi[r]);
        v.off[r] = off;
        v.row_off[r] = row;
        off += v.dlo[r] * v.dhi[r];
        row += v.dhi[r];
        v.blk_of_khi[khi[r]] = (int8_t)r;
    }
    v.off[nb] = off;
    v.row_off[nb] = row;
    v.dim = off;
    v.nrows = row;
}

}  // namespace ps
