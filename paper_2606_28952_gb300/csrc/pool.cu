// pool.cu -- energy gradients of a whole operator pool in one pass (the
// operator-selection step of ADAPT-VQE, Sec. 3.3).
//
// For every Hermitian single-X-group generator G_k of the pool,
//   g_k = d/dtheta <psi| e^{i theta G_k} H e^{-i theta G_k} |psi> at theta = 0
//       = i <psi|[G_k, H]|psi> = 2 Im <H psi | G_k psi>,
// which equals <psi|[H, A_k]|psi> for the anti-Hermitian A_k = -i G_k of the
// paper's notation.  H psi is given (it is the vector pauli_expect stores), so
// each g_k is one contraction of the same gather family: on a pair {t, s = t ^ x}
//   (G psi)_t = f_t psi_s,  (G psi)_s = conj(f_t) psi_t,
//   f_t = sum_{j in G} C_j (-1)^popcount(z_j & s).
// Generators that have pair lists on a single-block sector (rotation_pairs) are
// contracted together in one launch over (generator, pair range) work units;
// the others (full space, several blocks, x = 0) by a per-target kernel each.
// Every unit writes one FP64 partial; a fixed-order reduction per generator
// gives the K gradients (deterministic).
#include <algorithm>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {
namespace {

constexpr int kPoolPairsPerThread = 4;
constexpr int64_t kPoolPairs = (int64_t)kThreads * kPoolPairsPerThread;  // pairs per work unit

struct PoolDesc {
    const uint32_t *tab;     // pat_lo, rt_lo, rs_lo [nlo] each, then pat_hi, rt_hi, rs_hi [nhi]
    int64_t nlo, nhi;
    int64_t unit0, nunits;   // slice of the partial buffer
    uint64_t x;
    const uint64_t *z;       // [m]
    const double2 *c;        // [m]
    int m;
    int pad;
};

// contributions of one pair to <lam|G|phi>: conj(la) f b + conj(lb) conj(f) a
template <typename R>
__device__ __forceinline__ void pair_dot(DotAcc<R> &dot, R fr, R fi, const typename Cx<R>::T &a,
                                         const typename Cx<R>::T &b, const typename Cx<R>::T &la,
                                         const typename Cx<R>::T &lb) {
    typename Cx<R>::T fb, fa;
    fb.x = fr * b.x - fi * b.y;
    fb.y = fr * b.y + fi * b.x;
    fa.x = fr * a.x + fi * a.y;
    fa.y = fr * a.y - fi * a.x;
    dot.add(la, fb);
    dot.add(lb, fa);
}

template <typename R>
__device__ __forceinline__ void block_store_dot(const DotAcc<R> &dot, double *out2) {
    __shared__ double red[2][kThreads / 32];
    double mr = dot.get_re(), mi = dot.get_im();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mr += __shfl_down_sync(0xffffffffu, mr, o);
        mi += __shfl_down_sync(0xffffffffu, mi, o);
    }
    const int tid = threadIdx.x;
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = mr;
        red[1][tid >> 5] = mi;
    }
    __syncthreads();
    if (tid < 2) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += red[tid][w];
        out2[tid] = acc;
    }
}

// One CTA per work unit of the pair-listed generators.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_pool_pairs(const PoolDesc *__restrict__ descs, int ngen, int n_lo, int64_t off, int64_t dlo,
             const typename Cx<R>::T *__restrict__ psi, const typename Cx<R>::T *__restrict__ hpsi,
             double *__restrict__ partials) {
    using C2 = typename Cx<R>::T;
    __shared__ uint64_t sm_z[kRotPairTerms];
    __shared__ C2 sm_c[kRotPairTerms];
    const int64_t u = blockIdx.x;
    int lo = 0, hi = ngen - 1;  // last generator with unit0 <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (descs[mid].unit0 <= u) lo = mid;
        else hi = mid - 1;
    }
    const PoolDesc d = descs[lo];
    const int tid = threadIdx.x;
    for (int k = tid; k < d.m; k += kThreads) {
        sm_z[k] = d.z[k];
        const double2 cc = d.c[k];
        C2 cv;
        cv.x = (R)cc.x;
        cv.y = (R)cc.y;
        sm_c[k] = cv;
    }
    __syncthreads();
    const uint32_t *pat_lo = d.tab, *rt_lo = d.tab + d.nlo, *rs_lo = d.tab + 2 * d.nlo;
    const uint32_t *pat_hi = d.tab + 3 * d.nlo, *rt_hi = pat_hi + d.nhi, *rs_hi = pat_hi + 2 * d.nhi;
    const int64_t npairs = d.nlo * d.nhi;
    const int64_t p0 = (u - d.unit0) * kPoolPairs;
    DotAcc<R> dot;
#pragma unroll
    for (int j = 0; j < kPoolPairsPerThread; ++j) {
        const int64_t i = p0 + tid + (int64_t)j * kThreads;
        if (i >= npairs) break;
        const int64_t h = i / d.nlo, l = i - h * d.nlo;
        const uint64_t t = ((uint64_t)__ldg(pat_hi + h) << n_lo) | (uint64_t)__ldg(pat_lo + l);
        const uint64_t s = t ^ d.x;
        R fr = R(0), fi = R(0);
        for (int k = 0; k < d.m; ++k) {
            const uint32_t par = __popcll(sm_z[k] & s);
            fr += flip(sm_c[k].x, par);
            fi += flip(sm_c[k].y, par);
        }
        const int64_t it = off + (int64_t)__ldg(rt_hi + h) * dlo + __ldg(rt_lo + l);
        const int64_t is = off + (int64_t)__ldg(rs_hi + h) * dlo + __ldg(rs_lo + l);
        pair_dot<R>(dot, fr, fi, psi[it], psi[is], hpsi[it], hpsi[is]);
    }
    block_store_dot<R>(dot, partials + u * 2);
}

// Per-target contraction for one generator (full space, several blocks, x = 0):
// fixed grid, block-strided over the (row, column tile) units of the sector.
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_pool_generic(SectorView v, Geom geo, int64_t nwork, int64_t m, uint64_t x, const uint64_t *__restrict__ z,
               const double2 *__restrict__ c, const typename Cx<R>::T *__restrict__ psi,
               const typename Cx<R>::T *__restrict__ hpsi, double *__restrict__ partials, int *status) {
    using C2 = typename Cx<R>::T;
    __shared__ uint64_t sm_z[kRotPairTerms];
    __shared__ C2 sm_c[kRotPairTerms];
    const int tid = threadIdx.x;
    const uint32_t xlo = (uint32_t)(x & ((1ull << v.n_lo) - 1ull));
    const uint32_t xhi = (uint32_t)(x >> v.n_lo);
    DotAcc<R> dot;
    for (int64_t work = blockIdx.x; work < nwork; work += gridDim.x) {
        const RowCtx rc = decode_row<FULL>(v, geo, work);
        const int64_t col = rc.c0 + tid;
        const bool act = col < rc.dlo;
        uint32_t tlo = 0;
        if (act) tlo = FULL ? (uint32_t)col : __ldg(v.list_lo + v.lst_lo_off[rc.blk] + col);
        const uint32_t shi = rc.thi ^ xhi, slo = tlo ^ xlo;
        const uint64_t s = (uint64_t)slo | ((uint64_t)shi << v.n_lo);
        R fr = R(0), fi = R(0);
        for (int64_t k0 = 0; k0 < m; k0 += kRotPairTerms) {
            const int cnt = (m - k0 < kRotPairTerms) ? (int)(m - k0) : kRotPairTerms;
            __syncthreads();
            for (int k = tid; k < cnt; k += kThreads) {
                sm_z[k] = z[k0 + k];
                const double2 cc = c[k0 + k];
                C2 cv;
                cv.x = (R)cc.x;
                cv.y = (R)cc.y;
                sm_c[k] = cv;
            }
            __syncthreads();
            for (int k = 0; k < cnt; ++k) {
                const uint32_t par = __popcll(sm_z[k] & s);
                fr += flip(sm_c[k].x, par);
                fi += flip(sm_c[k].y, par);
            }
        }
        if (!act) continue;
        const int64_t tidx = rc.own_base + col;
        int64_t sidx;
        if (FULL) {
            sidx = (int64_t)s;
        } else {
            const int bb = v.blk_of_khi[cls_hi(v, shi)];
            if (bb < 0 || cls_lo(v, slo) != v.klo[bb]) {
                // P_S G P_S: a source outside the sector contributes nothing; record the leak
                if (fr != R(0) || fi != R(0)) atomicCAS(status, 0, (int)PAULI_ESECTOR);
                continue;
            }
            sidx = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb] + (int64_t)__ldg(v.rank_lo + slo);
        }
        if (x == 0) {
            // (G psi)_t = f_t psi_t
            C2 fa;
            const C2 a = psi[tidx];
            fa.x = fr * a.x - fi * a.y;
            fa.y = fr * a.y + fi * a.x;
            dot.add(hpsi[tidx], fa);
            continue;
        }
        if (tidx >= sidx) continue;  // each pair once, from its lower index
        pair_dot<R>(dot, fr, fi, psi[tidx], psi[sidx], hpsi[tidx], hpsi[sidx]);
    }
    block_store_dot<R>(dot, partials + (int64_t)blockIdx.x * 2);
}

// grads[k] = 2 Im (fixed-order sum of generator k's unit partials); range[2k],
// range[2k+1]: the generator's slice [first, end) of the partials
__global__ void __launch_bounds__(256) k_pool_reduce(const int64_t *__restrict__ range, const double *partials,
                                                     double *grads) {
    __shared__ double sm[256];
    const int k = blockIdx.x, t = threadIdx.x;
    const int64_t u0 = range[2 * k], u1 = range[2 * k + 1];
    double s = 0.0;
    for (int64_t u = u0 + t; u < u1; u += 256) s += partials[u * 2 + 1];
    sm[t] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) sm[t] += sm[t + o];
        __syncthreads();
    }
    if (t == 0) grads[k] = 2.0 * sm[0];
}

}  // namespace
}  // namespace ps

using namespace ps;

struct pauli_pool {
    uint32_t magic;
    Allocator al;
    int K = 0;
    SectorView v;                      // of the sector given at creation (its tables must outlive the pool)
    struct Generic {
        int k;
        int64_t unit0, nunits, m;
        uint64_t x;
        uint64_t *z;                   // pool-owned copies
        double2 *c;
        int *status;                   // the generator's status word (leaks)
    };
    std::vector<Generic> generic;
    std::vector<PoolDesc> h_desc;      // pair-listed generators, ascending unit0
    PoolDesc *d_desc = nullptr;
    int64_t pair_units = 0, total_units = 0;
    double *d_partials = nullptr;      // [total_units][2]
    int64_t *d_unit0 = nullptr;        // [2K] slice [first, end) of each generator, in pool order
    void *d_store = nullptr;           // pool-owned copies of pair tables, masks and coefficients
};

namespace {
constexpr uint32_t kPoolMagic = 0x50504f31u;  // "PPO1"

void free_pool(pauli_pool *p) {
    if (!p) return;
    dev_free(p->al, p->d_desc);
    dev_free(p->al, p->d_partials);
    dev_free(p->al, p->d_unit0);
    dev_free(p->al, p->d_store);
    p->magic = 0;
    delete p;
}
}  // namespace

extern "C" {

int pauli_pool_create(pauli_sum *const *Gs, int K, const pauli_sector *s, pauli_pool **out) {
    pauli_pool *p = nullptr;
    cudaStream_t st = nullptr;
    try {
        clear_error();
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(K >= 1 && K <= (1 << 20), PAULI_EINVAL, "K must be in 1..1048576");
        PS_CHECK(Gs != nullptr, PAULI_EINVAL, "Gs is NULL");
        PS_CHECK(s != nullptr && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        for (int k = 0; k < K; ++k) {
            PS_CHECK(Gs[k] != nullptr && Gs[k]->magic == kSumMagic, PAULI_EINVAL,
                     "pool: generator " + std::to_string(k) + " is not a valid pauli_sum handle");
            PS_CHECK(Gs[k]->n == s->v.n, PAULI_EINVAL, "pool: generator and sector qubit counts differ");
            PS_CHECK(Gs[k]->m == 0 || Gs[k]->G == 1, PAULI_EINVAL,
                     "pool: generator " + std::to_string(k) + " must have exactly one X mask");
            PS_CHECK(Gs[k]->hermitian, PAULI_ENOTHERMITIAN, "pool: generator " + std::to_string(k) + " is not Hermitian");
        }
        PS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        p = new pauli_pool();
        p->magic = kPoolMagic;
        p->al = current_allocator();
        p->K = K;
        p->v = s->v;
        // 1. classify; pair tables come from the generators' rotation caches
        struct Pend {
            int k;
            const RotPairs *rp;
            uint64_t x;
        };
        std::vector<Pend> pairs, gens;
        for (int k = 0; k < K; ++k) {
            pauli_sum *G = Gs[k];
            const uint64_t x = G->m ? group_mask0(G) : 0;
            const RotPairs *rp = G->m ? rotation_pairs(G, s, x, st) : nullptr;
            if (rp || G->m == 0) pairs.push_back({k, rp, x});
            else gens.push_back({k, nullptr, x});
        }
        // 2. pool-owned copies (tables, masks, coefficients): offsets in one buffer
        size_t bytes = 0;
        auto reserve = [&](size_t b) {
            const size_t at = bytes;
            bytes += (b + 255) & ~(size_t)255;
            return at;
        };
        std::vector<size_t> at_tab(K, 0), at_z(K, 0), at_c(K, 0);
        for (const Pend &q : pairs)
            if (q.rp) {
                at_tab[q.k] = reserve((size_t)3 * (q.rp->nlo + q.rp->nhi) * sizeof(uint32_t));
                at_z[q.k] = reserve((size_t)Gs[q.k]->m * 8);
                at_c[q.k] = reserve((size_t)Gs[q.k]->m * 16);
            }
        for (const Pend &q : gens) {
            at_z[q.k] = reserve((size_t)Gs[q.k]->m * 8);
            at_c[q.k] = reserve((size_t)Gs[q.k]->m * 16);
        }
        p->d_store = dev_alloc(p->al, bytes ? bytes : 256);
        char *base = static_cast<char *>(p->d_store);
        // 3. unit slices: pair-listed generators first, then the per-target ones
        std::vector<int64_t> unit0(K + 1, 0), nunits(K, 0);
        int64_t u = 0;
        for (const Pend &q : pairs) {
            pauli_sum *G = Gs[q.k];
            const int64_t np = q.rp ? q.rp->nlo * q.rp->nhi : 0;
            const int64_t nu = (np + kPoolPairs - 1) / kPoolPairs;
            unit0[q.k] = u;
            nunits[q.k] = nu;
            if (q.rp && nu > 0) {
                const size_t tb = (size_t)3 * (q.rp->nlo + q.rp->nhi) * sizeof(uint32_t);
                if (tb) PS_CUDA(cudaMemcpyAsync(base + at_tab[q.k], q.rp->tab, tb, cudaMemcpyDeviceToDevice, st));
                PS_CUDA(cudaMemcpyAsync(base + at_z[q.k], G->z, G->m * 8, cudaMemcpyDeviceToDevice, st));
                PS_CUDA(cudaMemcpyAsync(base + at_c[q.k], G->c, G->m * 16, cudaMemcpyDeviceToDevice, st));
                PoolDesc d;
                d.tab = reinterpret_cast<const uint32_t *>(base + at_tab[q.k]);
                d.nlo = q.rp->nlo;
                d.nhi = q.rp->nhi;
                d.unit0 = u;
                d.nunits = nu;
                d.x = q.x;
                d.z = reinterpret_cast<const uint64_t *>(base + at_z[q.k]);
                d.c = reinterpret_cast<const double2 *>(base + at_c[q.k]);
                d.m = (int)G->m;
                d.pad = 0;
                p->h_desc.push_back(d);
            }
            u += nu;
        }
        p->pair_units = u;
        const Geom geo = make_geom(s->v, kThreads);
        const int64_t nwork = geo.cta_off[s->v.nblk];
        const int64_t gen_units = std::max<int64_t>(1, std::min<int64_t>(nwork, (int64_t)num_sms() * 8));
        for (const Pend &q : gens) {
            pauli_sum *G = Gs[q.k];
            PS_CUDA(cudaMemcpyAsync(base + at_z[q.k], G->z, G->m * 8, cudaMemcpyDeviceToDevice, st));
            PS_CUDA(cudaMemcpyAsync(base + at_c[q.k], G->c, G->m * 16, cudaMemcpyDeviceToDevice, st));
            pauli_pool::Generic g;
            g.k = q.k;
            g.unit0 = u;
            g.nunits = nwork > 0 ? gen_units : 0;
            g.m = G->m;
            g.x = q.x;
            g.z = reinterpret_cast<uint64_t *>(base + at_z[q.k]);
            g.c = reinterpret_cast<double2 *>(base + at_c[q.k]);
            g.status = G->status;
            p->generic.push_back(g);
            unit0[q.k] = u;
            nunits[q.k] = g.nunits;
            u += g.nunits;
        }
        p->total_units = u;
        // each generator's slice [first, end) of the partials, in pool order
        std::vector<int64_t> ranges(2 * (size_t)K);
        for (int k = 0; k < K; ++k) {
            ranges[2 * k] = unit0[k];
            ranges[2 * k + 1] = unit0[k] + nunits[k];
        }
        p->d_unit0 = static_cast<int64_t *>(dev_alloc(p->al, ranges.size() * sizeof(int64_t)));
        PS_CUDA(cudaMemcpyAsync(p->d_unit0, ranges.data(), ranges.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        p->d_partials = static_cast<double *>(dev_alloc(p->al, (size_t)std::max<int64_t>(1, u) * 2 * sizeof(double)));
        if (!p->h_desc.empty()) {
            p->d_desc = static_cast<PoolDesc *>(dev_alloc(p->al, p->h_desc.size() * sizeof(PoolDesc)));
            PS_CUDA(cudaMemcpyAsync(p->d_desc, p->h_desc.data(), p->h_desc.size() * sizeof(PoolDesc),
                                    cudaMemcpyHostToDevice, st));
        }
        PS_CUDA(cudaStreamSynchronize(st));
        (void)cudaStreamDestroy(st);
        *out = p;
        return PAULI_OK;
    } catch (const Error &e) {
        if (st) {
            (void)cudaStreamSynchronize(st);
            (void)cudaStreamDestroy(st);
        }
        free_pool(p);
        set_error(e.msg);
        return e.code;
    } catch (...) {
        if (st) (void)cudaStreamDestroy(st);
        free_pool(p);
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_pool_size(const pauli_pool *p, int *K) {
    if (!p || p->magic != kPoolMagic || !K) {
        set_error("invalid pauli_pool handle or NULL K");
        return PAULI_EINVAL;
    }
    clear_error();
    *K = p->K;
    return PAULI_OK;
}

int pauli_pool_gradients(pauli_pool *p, const void *psi, const void *hpsi, int dtype, double *grads,
                         pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(p && p->magic == kPoolMagic, PAULI_EINVAL, "not a valid pauli_pool handle");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "dtype must be PAULI_C64 or PAULI_C128");
        PS_CHECK(psi && ((uintptr_t)psi % 16) == 0, PAULI_EINVAL, "psi is NULL or not 16-byte aligned");
        PS_CHECK(hpsi && ((uintptr_t)hpsi % 16) == 0, PAULI_EINVAL, "hpsi is NULL or not 16-byte aligned");
        PS_CHECK(grads != nullptr, PAULI_EINVAL, "grads is NULL");
        cudaStream_t cs = (cudaStream_t)st;
        const SectorView &v = p->v;
        if (p->pair_units > 0) {
            PS_CHECK(p->pair_units < (1ll << 31), PAULI_EUNSUPPORTED, "pool: too many work units");
            const int ng = (int)p->h_desc.size();
            if (dtype == PAULI_C64)
                k_pool_pairs<float><<<(unsigned)p->pair_units, kThreads, 0, cs>>>(
                    p->d_desc, ng, v.n_lo, v.off[0], v.dlo[0], static_cast<const float2 *>(psi),
                    static_cast<const float2 *>(hpsi), p->d_partials);
            else
                k_pool_pairs<double><<<(unsigned)p->pair_units, kThreads, 0, cs>>>(
                    p->d_desc, ng, v.n_lo, v.off[0], v.dlo[0], static_cast<const double2 *>(psi),
                    static_cast<const double2 *>(hpsi), p->d_partials);
            PS_LAUNCH_CHECK();
        }
        if (!p->generic.empty()) {
            const Geom geo = make_geom(v, kThreads);
            const int64_t nwork = geo.cta_off[v.nblk];
            const bool full = v.kind == PAULI_SECTOR_FULL;
            for (const pauli_pool::Generic &g : p->generic) {
                if (g.nunits == 0) continue;
                double *part = p->d_partials + g.unit0 * 2;
                const unsigned grid = (unsigned)g.nunits;
                if (dtype == PAULI_C64) {
                    auto *a = static_cast<const float2 *>(psi);
                    auto *b = static_cast<const float2 *>(hpsi);
                    if (full) k_pool_generic<float, true><<<grid, kThreads, 0, cs>>>(v, geo, nwork, g.m, g.x, g.z, g.c, a, b, part, g.status);
                    else k_pool_generic<float, false><<<grid, kThreads, 0, cs>>>(v, geo, nwork, g.m, g.x, g.z, g.c, a, b, part, g.status);
                } else {
                    auto *a = static_cast<const double2 *>(psi);
                    auto *b = static_cast<const double2 *>(hpsi);
                    if (full) k_pool_generic<double, true><<<grid, kThreads, 0, cs>>>(v, geo, nwork, g.m, g.x, g.z, g.c, a, b, part, g.status);
                    else k_pool_generic<double, false><<<grid, kThreads, 0, cs>>>(v, geo, nwork, g.m, g.x, g.z, g.c, a, b, part, g.status);
                }
                PS_LAUNCH_CHECK();
            }
        }
        k_pool_reduce<<<p->K, 256, 0, cs>>>(p->d_unit0, p->d_partials, grads);
        PS_LAUNCH_CHECK();
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_pool_destroy(pauli_pool *p) {
    if (!p) return PAULI_OK;
    if (p->magic != kPoolMagic) {
        set_error("not a valid pauli_pool handle");
        return PAULI_EINVAL;
    }
    clear_error();
    free_pool(p);
    return PAULI_OK;
}

}  // extern "C"
