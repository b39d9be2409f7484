// wide.cu -- Pauli sums on more than 64 qubits (multi-word X / Z masks):
// Jordan-Wigner construction (Algorithm 1, JW ladder strings of Sec. 2.3),
// canonical reduction (Sec. 2.3) and operator products (eq.
// pauli_operator_multiplication), with masks of W = ceil(n / 64) 64-bit
// words, n <= 256.  The state-vector kernels stay at n <= 64 (a state of more
// qubits does not fit any memory); this is the operator algebra of the paper's
// large Jordan-Wigner builds.
//
// Storage: term t has words x[t * W + w], z[t * W + w] (word w = qubits
// 64 w .. 64 w + 63) and an XZ-form coefficient c[t].  Canonical order: (x, z)
// ascending as unsigned multi-word integers, x first.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kWMax = 4;
constexpr int kWThreads = 256;
constexpr int kWRounds = 8;
constexpr int kWTile = kWThreads * kWRounds;
constexpr int kWWarps = kWThreads / 32;

struct WFactor {
    int P;
    int dag;
};

// JW raw entries of one product of ladder operators (left to right) with W-word
// masks: a_P^dagger = 1/2 X^{e_P} Z^{below} + 1/2 X^{e_P} Z^{below | e_P},
// a_P = 1/2 X^{e_P} Z^{below} - 1/2 X^{e_P} Z^{below | e_P} (XZ form), and
// (X^a Z^b)(X^c Z^d) = (-1)^popcount(b & c) X^(a ^ c) Z^(b ^ d).
template <int W>
__device__ void wexpand(const WFactor *f, int nf, double2 scale, int64_t pos, uint64_t *ox, uint64_t *oz,
                        double2 *oc) {
    const int ne = 1 << nf;
    for (int e = 0; e < ne; ++e) {
        uint64_t x[W], z[W];
#pragma unroll
        for (int w = 0; w < W; ++w) x[w] = z[w] = 0ull;
        int neg = 0;
        double mag = 1.0;
        for (int j = 0; j < nf; ++j) {
            const int sel = (e >> (nf - 1 - j)) & 1;
            const int P = f[j].P, wp = P >> 6;
            const uint64_t bit = 1ull << (P & 63);
            // phase from the Z part accumulated so far against the new X bit
            neg ^= (int)((z[wp] >> (P & 63)) & 1ull);
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t fz = w < wp ? ~0ull : (w == wp ? (bit - 1ull) | (sel ? bit : 0ull) : 0ull);
                z[w] ^= fz;
            }
            x[wp] ^= bit;
            if (sel && !f[j].dag) neg ^= 1;
            mag *= 0.5;
        }
        const double s = neg ? -mag : mag;
        for (int w = 0; w < W; ++w) {
            ox[(pos + e) * W + w] = x[w];
            oz[(pos + e) * W + w] = z[w];
        }
        oc[pos + e] = make_double2(scale.x * s, scale.y * s);
    }
}

template <int W>
__global__ void k_wfermion_expand(int64_t nterms, const int *nf, const int64_t *fstart, const int *modes,
                                  const int *dag, const double2 *coef, const int64_t *off, uint64_t *ox,
                                  uint64_t *oz, double2 *oc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nterms) return;
    WFactor f[8];
    for (int j = 0; j < nf[t]; ++j) f[j] = {modes[fstart[t] + j], dag[fstart[t] + j]};
    wexpand<W>(f, nf[t], coef[t], off[t], ox, oz, oc);
}

// raw entries of A B, pair (k, l) at k * mb + l: Ca Cb (-1)^popcount(za & xb)
template <int W>
__global__ void k_wproduct(int64_t ma, const uint64_t *xa, const uint64_t *za, const double2 *ca, int64_t mb,
                           const uint64_t *xb, const uint64_t *zb, const double2 *cb, uint64_t *ox, uint64_t *oz,
                           double2 *oc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ma * mb) return;
    const int64_t k = i / mb, l = i - k * mb;
    int par = 0;
    for (int w = 0; w < W; ++w) {
        const uint64_t x1 = xa[k * W + w], z1 = za[k * W + w], x2 = xb[l * W + w], z2 = zb[l * W + w];
        par ^= __popcll(z1 & x2) & 1;
        ox[i * W + w] = x1 ^ x2;
        oz[i * W + w] = z1 ^ z2;
    }
    const double2 a = ca[k], b = cb[l];
    double re = __dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
    double im = __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x));
    if (par) {
        re = -re;
        im = -im;
    }
    oc[i] = make_double2(re, im);
}

__global__ void k_widx(int64_t *p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

// digit (8 bits at `shift`) of word `w` of key perm[i]; key words: z words
// then x words (LSD order: z[0] least significant)
__device__ __forceinline__ int wdigit(const uint64_t *x, const uint64_t *z, int W, int64_t t, int kw, int shift) {
    const uint64_t v = kw < W ? z[t * W + kw] : x[t * W + (kw - W)];
    return (int)((v >> shift) & 255ull);
}

__global__ void k_whist(const uint64_t *x, const uint64_t *z, int W, const int64_t *perm, int64_t n, int kw,
                        int shift, int64_t ntiles, int64_t *hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kWTile;
    for (int r = 0; r < kWRounds; ++r) {
        const int64_t i = base + r * kWThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[wdigit(x, z, W, perm[i], kw, shift)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// stable scatter of the permutation by the digit (warp match ranks, in-order rounds)
__global__ void k_wscatter(const uint64_t *x, const uint64_t *z, int W, const int64_t *perm, int64_t n, int kw,
                           int shift, int64_t ntiles, const int64_t *offs, int64_t *operm) {
    __shared__ int wcount[kWWarps][256];
    __shared__ int64_t base_cnt[256];
    __shared__ int round_tot[256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int w = 0; w < kWWarps; ++w) wcount[w][t] = 0;
    base_cnt[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t tile0 = (int64_t)blockIdx.x * kWTile;
    for (int r = 0; r < kWRounds; ++r) {
        const int64_t i = tile0 + r * kWThreads + t;
        const bool valid = i < n;
        int64_t p = 0;
        int d = 256 + lane;
        if (valid) {
            p = perm[i];
            d = wdigit(x, z, W, p, kw, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank_in_warp = __popc(peers & lt_mask);
        if (valid && rank_in_warp == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {
            int pre = 0;
            for (int w = 0; w < kWWarps; ++w) {
                const int c = wcount[w][t];
                wcount[w][t] = pre;
                pre += c;
            }
            round_tot[t] = pre;
        }
        __syncthreads();
        if (valid) operm[base_cnt[d] + wcount[warp][d] + rank_in_warp] = p;
        __syncthreads();
        base_cnt[t] += round_tot[t];
        for (int w = 0; w < kWWarps; ++w) wcount[w][t] = 0;
        __syncthreads();
    }
}

// 1 where sorted key i differs from key i - 1 (x only if xonly)
__global__ void k_wheads(const uint64_t *x, const uint64_t *z, int W, const int64_t *perm, int64_t n, int xonly,
                         int64_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0) {
        flag[0] = 1;
        return;
    }
    const int64_t a = perm ? perm[i] : i, b = perm ? perm[i - 1] : i - 1;
    int diff = 0;
    for (int w = 0; w < W; ++w) {
        diff |= x[a * W + w] != x[b * W + w];
        if (!xonly) diff |= z[a * W + w] != z[b * W + w];
    }
    flag[i] = diff;
}

__global__ void k_wstarts(const int64_t *flag, const int64_t *id, int64_t n, int64_t *start) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) start[id[i]] = i;
}

// one thread per run: left-to-right sum in input order (the sort is stable), drop test
__global__ void k_wsums(int64_t nruns, int64_t n, const int64_t *start, const int64_t *perm, const double2 *c,
                        double eps2, double2 *sum, int64_t *keep) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    const int64_t a = start[r], b = (r + 1 < nruns) ? start[r + 1] : n;
    double2 s = c[perm[a]];
    for (int64_t j = a + 1; j < b; ++j) {
        const double2 v = c[perm[j]];
        s.x = __dadd_rn(s.x, v.x);
        s.y = __dadd_rn(s.y, v.y);
    }
    sum[r] = s;
    keep[r] = __dadd_rn(__dmul_rn(s.x, s.x), __dmul_rn(s.y, s.y)) > eps2 ? 1 : 0;
}

__global__ void k_wcompact(int64_t nruns, int W, const int64_t *start, const int64_t *keep, const int64_t *pos,
                           const int64_t *perm, const uint64_t *x, const uint64_t *z, const double2 *sum, uint64_t *ox,
                           uint64_t *oz, double2 *oc) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns || !keep[r]) return;
    const int64_t o = pos[r], src = perm[start[r]];
    for (int w = 0; w < W; ++w) {
        ox[o * W + w] = x[src * W + w];
        oz[o * W + w] = z[src * W + w];
    }
    oc[o] = sum[r];
}

unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

int64_t last_of(const int64_t *d, int64_t n, cudaStream_t st) {
    int64_t v = 0;
    PS_CUDA(cudaMemcpyAsync(&v, d + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    return v;
}

}  // namespace
}  // namespace ps

using namespace ps;

struct pauli_wsum {
    uint32_t magic;
    Allocator al;
    int n = 0, W = 1;
    int64_t m = 0, G = 0;
    uint64_t *x = nullptr, *z = nullptr;  // [m * W]
    double2 *c = nullptr;                  // [m]
    int64_t *gstart = nullptr;             // [G + 1]
};

namespace {
constexpr uint32_t kWSumMagic = 0x50575331u;  // "PWS1"

void free_wsum(pauli_wsum *h) {
    if (!h) return;
    dev_free(h->al, h->x);
    dev_free(h->al, h->z);
    dev_free(h->al, h->c);
    dev_free(h->al, h->gstart);
    h->magic = 0;
    delete h;
}

struct WGuard {
    pauli_wsum *h;
    ~WGuard() { free_wsum(h); }
    pauli_wsum *release() {
        pauli_wsum *p = h;
        h = nullptr;
        return p;
    }
};

pauli_wsum *new_wsum(int n) {
    auto h = new pauli_wsum();
    h->magic = kWSumMagic;
    h->al = current_allocator();
    h->n = n;
    h->W = (n + 63) / 64;
    return h;
}

// canonical reduction of m raw entries (device arrays, x / z with h->W words)
void wcanonical(pauli_wsum *h, int64_t m, const uint64_t *x, const uint64_t *z, const double2 *c, double eps,
                cudaStream_t st) {
    const Allocator &al = h->al;
    const int W = h->W;
    h->m = h->G = 0;
    if (m > 0) {
        DevBuf<int64_t> perm(al, m), perm2(al, m);
        k_widx<<<nb(m), 256, 0, st>>>(perm.p, m);
        PS_LAUNCH_CHECK();
        const int64_t ntiles = (m + kWTile - 1) / kWTile;
        DevBuf<int64_t> hist(al, 256 * ntiles), offs(al, 256 * ntiles);
        int64_t *cp = perm.p, *np = perm2.p;
        // LSD: z words (least significant first), then x words; bits above n skipped
        for (int kw = 0; kw < 2 * W; ++kw) {
            const int w = kw % W;
            const int bits = std::min(64, h->n - 64 * w);
            for (int shift = 0; shift < bits; shift += 8) {
                k_whist<<<(unsigned)ntiles, kWThreads, 0, st>>>(x, z, W, cp, m, kw, shift, ntiles, hist.p);
                PS_LAUNCH_CHECK();
                exclusive_scan_i64(hist.p, offs.p, 256 * ntiles, al, st);
                k_wscatter<<<(unsigned)ntiles, kWThreads, 0, st>>>(x, z, W, cp, m, kw, shift, ntiles, offs.p, np);
                PS_LAUNCH_CHECK();
                std::swap(cp, np);
            }
        }
        DevBuf<int64_t> flag(al, m), id(al, m);
        k_wheads<<<nb(m), 256, 0, st>>>(x, z, W, cp, m, 0, flag.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(flag.p, id.p, m, al, st);
        const int64_t nruns = last_of(id.p, m, st) + last_of(flag.p, m, st);
        DevBuf<int64_t> start(al, nruns), keep(al, nruns), pos(al, nruns);
        DevBuf<double2> sum(al, nruns);
        k_wstarts<<<nb(m), 256, 0, st>>>(flag.p, id.p, m, start.p);
        PS_LAUNCH_CHECK();
        k_wsums<<<nb(nruns), 256, 0, st>>>(nruns, m, start.p, cp, c, eps * eps, sum.p, keep.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(keep.p, pos.p, nruns, al, st);
        const int64_t M = last_of(pos.p, nruns, st) + last_of(keep.p, nruns, st);
        h->m = M;
        h->x = static_cast<uint64_t *>(dev_alloc(al, std::max<int64_t>(1, M) * W * 8));
        h->z = static_cast<uint64_t *>(dev_alloc(al, std::max<int64_t>(1, M) * W * 8));
        h->c = static_cast<double2 *>(dev_alloc(al, std::max<int64_t>(1, M) * 16));
        k_wcompact<<<nb(nruns), 256, 0, st>>>(nruns, W, start.p, keep.p, pos.p, cp, x, z, sum.p, h->x, h->z, h->c);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaStreamSynchronize(st));
    }
    if (!h->x) {
        h->x = static_cast<uint64_t *>(dev_alloc(al, W * 8));
        h->z = static_cast<uint64_t *>(dev_alloc(al, W * 8));
        h->c = static_cast<double2 *>(dev_alloc(al, 16));
    }
    // X-mask groups: runs of equal x in the canonical order
    const int64_t M = h->m;
    if (M > 0) {
        DevBuf<int64_t> flag(al, M), id(al, M);
        k_wheads<<<nb(M), 256, 0, st>>>(h->x, h->z, W, nullptr, M, 1, flag.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(flag.p, id.p, M, al, st);
        const int64_t G = last_of(id.p, M, st) + last_of(flag.p, M, st);
        h->G = G;
        h->gstart = static_cast<int64_t *>(dev_alloc(al, (G + 1) * 8));
        k_wstarts<<<nb(M), 256, 0, st>>>(flag.p, id.p, M, h->gstart);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaMemcpyAsync(h->gstart + G, &M, 8, cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaStreamSynchronize(st));
    } else {
        h->gstart = static_cast<int64_t *>(dev_alloc(al, 8));
        PS_CUDA(cudaMemsetAsync(h->gstart, 0, 8, st));
        PS_CUDA(cudaStreamSynchronize(st));
    }
}

// Raw JW entries of fermionic monomials (host description) -> device arrays
void wfermion_raw(int W, int64_t nterms, const std::vector<int> &nf, const std::vector<int64_t> &fstart,
                  const std::vector<int> &modes, const std::vector<int> &dag, const std::vector<double2> &coef,
                  const Allocator &al, DevBuf<uint64_t> &x, DevBuf<uint64_t> &z, DevBuf<double2> &c, int64_t &count,
                  cudaStream_t st) {
    std::vector<int64_t> off(nterms, 0);
    count = 0;
    for (int64_t t = 0; t < nterms; ++t) {
        off[t] = count;
        count += (int64_t)1 << nf[t];
    }
    x = DevBuf<uint64_t>(al, (size_t)std::max<int64_t>(1, count) * W);
    z = DevBuf<uint64_t>(al, (size_t)std::max<int64_t>(1, count) * W);
    c = DevBuf<double2>(al, (size_t)std::max<int64_t>(1, count));
    if (nterms == 0) return;
    DevBuf<int> d_nf(al, nterms), d_modes(al, modes.size()), d_dag(al, dag.size());
    DevBuf<int64_t> d_fs(al, nterms + 1), d_off(al, nterms);
    DevBuf<double2> d_c(al, nterms);
    PS_CUDA(cudaMemcpyAsync(d_nf.p, nf.data(), nterms * sizeof(int), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(d_fs.p, fstart.data(), (nterms + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!modes.empty()) {
        PS_CUDA(cudaMemcpyAsync(d_modes.p, modes.data(), modes.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaMemcpyAsync(d_dag.p, dag.data(), dag.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    PS_CUDA(cudaMemcpyAsync(d_c.p, coef.data(), nterms * sizeof(double2), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(d_off.p, off.data(), nterms * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    switch (W) {
        case 1: k_wfermion_expand<1><<<nb(nterms), 256, 0, st>>>(nterms, d_nf.p, d_fs.p, d_modes.p, d_dag.p, d_c.p, d_off.p, x.p, z.p, c.p); break;
        case 2: k_wfermion_expand<2><<<nb(nterms), 256, 0, st>>>(nterms, d_nf.p, d_fs.p, d_modes.p, d_dag.p, d_c.p, d_off.p, x.p, z.p, c.p); break;
        case 3: k_wfermion_expand<3><<<nb(nterms), 256, 0, st>>>(nterms, d_nf.p, d_fs.p, d_modes.p, d_dag.p, d_c.p, d_off.p, x.p, z.p, c.p); break;
        default: k_wfermion_expand<4><<<nb(nterms), 256, 0, st>>>(nterms, d_nf.p, d_fs.p, d_modes.p, d_dag.p, d_c.p, d_off.p, x.p, z.p, c.p); break;
    }
    PS_LAUNCH_CHECK();
    PS_CUDA(cudaStreamSynchronize(st));
}

template <typename F>
int wguarded(F &&f) {
    try {
        clear_error();
        f();
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return PAULI_ENOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

struct WStream {
    cudaStream_t s = nullptr;
    WStream() { PS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
    ~WStream() {
        if (s) {
            (void)cudaStreamSynchronize(s);
            (void)cudaStreamDestroy(s);
        }
    }
};

void check_wsum(const pauli_wsum *h) {
    PS_CHECK(h != nullptr && h->magic == kWSumMagic, PAULI_EINVAL, "not a valid pauli_wsum handle");
}

}  // namespace

extern "C" {

int pauli_wsum_jw_fermion(int n_qubits, int n_terms, const int *n_factors, const int *modes, const int *daggers,
                          const double *c_re, const double *c_im, double eps_drop, pauli_wsum **out) {
    return wguarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n_qubits >= 1 && n_qubits <= 64 * kWMax, PAULI_EINVAL, "n_qubits must be in 1..256");
        PS_CHECK(n_terms >= 0, PAULI_EINVAL, "n_terms must be >= 0");
        PS_CHECK(n_terms == 0 || (n_factors && c_re && c_im), PAULI_EINVAL, "term arrays must not be NULL");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        std::vector<int> nf(n_terms), md, dg;
        std::vector<int64_t> fs(n_terms + 1, 0);
        std::vector<double2> cf(n_terms);
        for (int t = 0; t < n_terms; ++t) {
            PS_CHECK(n_factors[t] >= 1 && n_factors[t] <= 8, PAULI_EINVAL, "each term needs 1..8 factors");
            PS_CHECK(std::isfinite(c_re[t]) && std::isfinite(c_im[t]), PAULI_EINVAL, "non-finite coefficient");
            nf[t] = n_factors[t];
            fs[t + 1] = fs[t] + nf[t];
            cf[t] = make_double2(c_re[t], c_im[t]);
        }
        PS_CHECK(fs[n_terms] == 0 || (modes && daggers), PAULI_EINVAL, "modes / daggers must not be NULL");
        for (int64_t j = 0; j < fs[n_terms]; ++j) {
            PS_CHECK(modes[j] >= 0 && modes[j] < n_qubits, PAULI_EINVAL, "mode index out of range");
            md.push_back(modes[j]);
            dg.push_back(daggers[j] ? 1 : 0);
        }
        WStream st;
        WGuard g{new_wsum(n_qubits)};
        DevBuf<uint64_t> x, z;
        DevBuf<double2> c;
        int64_t cnt = 0;
        wfermion_raw(g.h->W, n_terms, nf, fs, md, dg, cf, g.h->al, x, z, c, cnt, st.s);
        wcanonical(g.h, cnt, x.p, z.p, c.p, eps_drop, st.s);
        *out = g.release();
    });
}

int pauli_wsum_jw_molecular(int n_orb, const double *h, const double *g, double e_nn, double eps_int,
                            double eps_drop, pauli_wsum **out) {
    return wguarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n_orb >= 1 && n_orb <= 32 * kWMax, PAULI_EINVAL, "n_orb must be in 1..128");
        PS_CHECK(h && g, PAULI_EINVAL, "integral arrays must not be NULL");
        PS_CHECK(std::isfinite(e_nn) && std::isfinite(eps_int) && eps_int >= 0.0 && std::isfinite(eps_drop) &&
                     eps_drop >= 0.0,
                 PAULI_EINVAL, "e_nn, eps_int and eps_drop must be finite (and the thresholds >= 0)");
        const int64_t n2 = (int64_t)n_orb * n_orb, n4 = n2 * n2;
        for (int64_t i = 0; i < n2; ++i) PS_CHECK(std::isfinite(h[i]), PAULI_EINVAL, "h has a non-finite entry");
        for (int64_t i = 0; i < n4; ++i) PS_CHECK(std::isfinite(g[i]), PAULI_EINVAL, "g has a non-finite entry");
        // Algorithm 1's raw order as monomials: the e_nn identity, one-body
        // h_pq a+_{ps} a_{qs} (s, p, q ascending), two-body
        // 1/2 (pq|ru) a+_{ps} a+_{rt} a_{ut} a_{qs} (s, t, p, q, r, u ascending),
        // skipping |v| <= eps_int and P == R or Q == U
        std::vector<int> nf, md, dg;
        std::vector<int64_t> fs(1, 0);
        std::vector<double2> cf;
        auto add = [&](std::initializer_list<std::pair<int, int>> f, double v) {
            for (auto &e : f) {
                md.push_back(e.first);
                dg.push_back(e.second);
            }
            nf.push_back((int)f.size());
            fs.push_back(fs.back() + (int64_t)f.size());
            cf.push_back(make_double2(v, 0.0));
        };
        const int n = 2 * n_orb;
        // the identity entry: the empty product is not a monomial here, so it is
        // added after the expansion as its own raw entry in front
        for (int s = 0; s < 2; ++s)
            for (int p = 0; p < n_orb; ++p)
                for (int q = 0; q < n_orb; ++q) {
                    const double v = h[p * n_orb + q];
                    if (std::fabs(v) > eps_int) add({{s * n_orb + p, 1}, {s * n_orb + q, 0}}, v);
                }
        for (int s = 0; s < 2; ++s)
            for (int t = 0; t < 2; ++t)
                for (int p = 0; p < n_orb; ++p)
                    for (int q = 0; q < n_orb; ++q)
                        for (int r = 0; r < n_orb; ++r)
                            for (int u = 0; u < n_orb; ++u) {
                                const double v = g[(((int64_t)p * n_orb + q) * n_orb + r) * n_orb + u];
                                if (!(std::fabs(v) > eps_int)) continue;
                                const int P = s * n_orb + p, Q = s * n_orb + q, R = t * n_orb + r, U = t * n_orb + u;
                                if (P == R || Q == U) continue;
                                add({{P, 1}, {R, 1}, {U, 0}, {Q, 0}}, 0.5 * v);
                            }
        WStream st;
        WGuard gd{new_wsum(n)};
        const int W = gd.h->W;
        DevBuf<uint64_t> x, z;
        DevBuf<double2> c;
        int64_t cnt = 0;
        const int64_t nt = (int64_t)nf.size();
        wfermion_raw(W, nt, nf, fs, md, dg, cf, gd.h->al, x, z, c, cnt, st.s);
        if (e_nn != 0.0) {
            // prepend the identity entry (raw order: e_nn first)
            DevBuf<uint64_t> x2(gd.h->al, (size_t)(cnt + 1) * W), z2(gd.h->al, (size_t)(cnt + 1) * W);
            DevBuf<double2> c2(gd.h->al, (size_t)cnt + 1);
            PS_CUDA(cudaMemsetAsync(x2.p, 0, W * 8, st.s));
            PS_CUDA(cudaMemsetAsync(z2.p, 0, W * 8, st.s));
            const double2 ce = make_double2(e_nn, 0.0);
            PS_CUDA(cudaMemcpyAsync(c2.p, &ce, 16, cudaMemcpyHostToDevice, st.s));
            if (cnt > 0) {
                PS_CUDA(cudaMemcpyAsync(x2.p + W, x.p, cnt * W * 8, cudaMemcpyDeviceToDevice, st.s));
                PS_CUDA(cudaMemcpyAsync(z2.p + W, z.p, cnt * W * 8, cudaMemcpyDeviceToDevice, st.s));
                PS_CUDA(cudaMemcpyAsync(c2.p + 1, c.p, cnt * 16, cudaMemcpyDeviceToDevice, st.s));
            }
            PS_CUDA(cudaStreamSynchronize(st.s));
            x = std::move(x2);
            z = std::move(z2);
            c = std::move(c2);
            ++cnt;
        }
        wcanonical(gd.h, cnt, x.p, z.p, c.p, eps_drop, st.s);
        *out = gd.release();
    });
}

int pauli_wsum_product(const pauli_wsum *A, const pauli_wsum *B, double eps_drop, pauli_wsum **out) {
    return wguarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        check_wsum(A);
        check_wsum(B);
        PS_CHECK(A->n == B->n, PAULI_EINVAL, "operands have different qubit counts");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        const int64_t m = A->m * B->m;
        PS_CHECK(A->m == 0 || m / A->m == B->m, PAULI_EUNSUPPORTED, "product too large");
        PS_CHECK(m <= (1ll << 30), PAULI_EUNSUPPORTED, "product: more than 2^30 raw term pairs");
        WStream st;
        WGuard g{new_wsum(A->n)};
        const int W = g.h->W;
        DevBuf<uint64_t> x(g.h->al, (size_t)std::max<int64_t>(1, m) * W), z(g.h->al, (size_t)std::max<int64_t>(1, m) * W);
        DevBuf<double2> c(g.h->al, (size_t)std::max<int64_t>(1, m));
        if (m > 0) {
            switch (W) {
                case 1: k_wproduct<1><<<nb(m), 256, 0, st.s>>>(A->m, A->x, A->z, A->c, B->m, B->x, B->z, B->c, x.p, z.p, c.p); break;
                case 2: k_wproduct<2><<<nb(m), 256, 0, st.s>>>(A->m, A->x, A->z, A->c, B->m, B->x, B->z, B->c, x.p, z.p, c.p); break;
                case 3: k_wproduct<3><<<nb(m), 256, 0, st.s>>>(A->m, A->x, A->z, A->c, B->m, B->x, B->z, B->c, x.p, z.p, c.p); break;
                default: k_wproduct<4><<<nb(m), 256, 0, st.s>>>(A->m, A->x, A->z, A->c, B->m, B->x, B->z, B->c, x.p, z.p, c.p); break;
            }
            PS_LAUNCH_CHECK();
        }
        wcanonical(g.h, m, x.p, z.p, c.p, eps_drop, st.s);
        *out = g.release();
    });
}

int pauli_wsum_info(const pauli_wsum *h, int *n_qubits, int *words, int64_t *m, int64_t *n_groups) {
    return wguarded([&] {
        check_wsum(h);
        if (n_qubits) *n_qubits = h->n;
        if (words) *words = h->W;
        if (m) *m = h->m;
        if (n_groups) *n_groups = h->G;
    });
}

int pauli_wsum_export(const pauli_wsum *h, uint64_t *x, uint64_t *z, double *c_re, double *c_im) {
    return wguarded([&] {
        check_wsum(h);
        if (h->m == 0) return;
        PS_CHECK(x && z && c_re && c_im, PAULI_EINVAL, "output arrays must not be NULL");
        std::vector<double2> hc(h->m);
        PS_CUDA(cudaMemcpy(x, h->x, h->m * h->W * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(z, h->z, h->m * h->W * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(hc.data(), h->c, h->m * 16, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < h->m; ++i) {
            c_re[i] = hc[i].x;
            c_im[i] = hc[i].y;
        }
    });
}

int pauli_wsum_groups(const pauli_wsum *h, int64_t *group_start) {
    return wguarded([&] {
        check_wsum(h);
        PS_CHECK(group_start != nullptr, PAULI_EINVAL, "group_start is NULL");
        PS_CUDA(cudaMemcpy(group_start, h->gstart, (h->G + 1) * 8, cudaMemcpyDeviceToHost));
    });
}

int pauli_wsum_destroy(pauli_wsum *h) {
    return wguarded([&] {
        if (!h) return;
        check_wsum(h);
        free_wsum(h);
    });
}

}  // extern "C"
