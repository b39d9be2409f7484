// local.cu -- the full-space apply in passes over local bit sets.
//
// For an operator whose X masks touch few bits each (lattice models: bonds,
// plaquettes), the groups are split into passes such that every X mask of a
// pass lies inside one set L of kLocBits bit positions that always contains
// the kLocRun lowest bits.  A CTA owns one chunk: the 2^kLocBits amplitudes
// that share the bits outside L.  It stages the chunk in shared memory (runs of
// 2^kLocRun contiguous amplitudes), folds the phases of the bits outside L into
// the term coefficients once, and gathers every source of eq. reverse_sum for
// the pass's groups from shared memory.  The first pass writes H psi, later
// passes add to it in a fixed order (no atomics); the last one also produces
// the FP64 expectation partials.  The x = 0 group's terms without bits outside
// L come from a table over L.
//
// Clustered windows (LocalPlan::cb = 3): a pass's window of kLocBits + 3 bits is
// held by a cluster of 8 CTAs, each with the chunk of one value of the 3
// cluster bits; a group whose X mask has cluster bits reads its sources from
// the peer CTA's chunk through distributed shared memory.  Runs shrink to 2
// amplitudes (16 bytes) so that a 30-site chain needs two passes instead of three.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>

#include "apply_kernels.cuh"

namespace cg = cooperative_groups;

namespace ps {

namespace {

struct LocalPassDev {
    int b, m, nn;                  // local bits, high local bits (b - run), non-local bits
    int run;                       // log2 of the contiguous amplitudes of one staged run
    int cb;                        // cluster bits (0: one CTA per window)
    int g0, g1;                    // groups of the pass
    int diag;                      // 1: group g0 is the x = 0 group, tabulated
    int8_t npos[64];               // non-local bit positions: the cluster bits, then the rest ascending
    const uint64_t *hoff;          // [2^m] global offsets of the high local bits
};

struct LocalArgs {
    const uint32_t *g_xloc;   // [G'] x compressed to the pass's local bits
    const uint32_t *g_xcl;    // [G'] x on the cluster bits (the peer CTA's rank offset)
    const uint64_t *t_xnl;    // [M'] x of the term's group outside the CTA's local bits
    const int32_t *g_t0;      // [G'+1] terms of each group
    const int32_t *g_tz;      // [G'] end of the group's terms with z_loc = 0
    const uint32_t *t_zloc;   // [M'] z compressed to the local bits
    const uint64_t *t_znl;    // [M'] z outside the local bits (global positions)
    const double2 *t_c;       // [M'] coefficients
    const double2 *dtab64;    // [2^b] table of the x = 0 group's terms with z_nl = 0
    const float2 *dtab32;     // [2 * 2^b] the same, FP32 hi then lo
};

template <typename R>
__device__ __forceinline__ typename Cx<R>::T ld_tab(const LocalArgs &a, uint32_t l, uint32_t n, R &lo_re, R &lo_im);
template <>
__device__ __forceinline__ float2 ld_tab<float>(const LocalArgs &a, uint32_t l, uint32_t n, float &lo_re, float &lo_im) {
    const float2 lo = __ldg(a.dtab32 + n + l);
    lo_re = lo.x;
    lo_im = lo.y;
    return __ldg(a.dtab32 + l);
}
template <>
__device__ __forceinline__ double2 ld_tab<double>(const LocalArgs &a, uint32_t l, uint32_t, double &lo_re,
                                                  double &lo_im) {
    lo_re = 0.0;
    lo_im = 0.0;
    return __ldg(a.dtab64 + l);
}

template <typename R, bool REALH, int TPT>
__global__ void __launch_bounds__(kThreads)
k_apply_local(LocalPassDev P, LocalArgs A, const typename Cx<R>::T *__restrict__ psi,
              typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    using C2 = typename Cx<R>::T;
    constexpr int kEShift = sizeof(C2) == 8 ? 3 : 4;  // log2 of the amplitude size
    extern __shared__ __align__(16) char smem[];
    const int nloc = 1 << P.b;
    const int ng = P.g1 - P.g0;
    const int t_first = A.g_t0[P.g0], t_last = A.g_t0[P.g1];
    const int nt = t_last - t_first;
    // layout: chunk (2^b amplitudes, a multiple of 16 bytes), group records (16 B
    // each), folded coefficients, per-group constants, z masks
    C2 *chunk = reinterpret_cast<C2 *>(smem);
    int4 *sm_g = reinterpret_cast<int4 *>(chunk + nloc);          // [ng] {x_loc, first, end} of the z_loc != 0 terms
    C2 *sm_c = reinterpret_cast<C2 *>(sm_g + ng);                 // [nt] folded coefficients
    C2 *sm_a0 = sm_c + nt;                                        // [ng] sums of the z_loc = 0 terms
    uint32_t *sm_z = reinterpret_cast<uint32_t *>(sm_a0 + ng);     // [nt]
    const int tid = threadIdx.x;
    // global bits of this chunk
    uint64_t base = 0;
    {
        uint64_t k = blockIdx.x;
        for (int i = 0; i < P.nn; ++i, k >>= 1) base |= (k & 1ull) << P.npos[i];
    }
    // this CTA's rank in its cluster: the cluster bits are the lowest of blockIdx.x
    const uint32_t rank = blockIdx.x & ((1u << P.cb) - 1u);
    // 1. the chunk -> shared memory, 16-byte copies (runs of 2^run amplitudes)
    constexpr int kPerCopy = 16 / (int)sizeof(C2);  // amplitudes per 16-byte copy
    const int lrun = P.run;
    const int crun = (1 << lrun) / kPerCopy;        // copies per run (a power of two)
    const int lcrun = __ffs(crun) - 1;
    const int ncopy = nloc / kPerCopy;
    for (int u = tid; u < ncopy; u += kThreads) {
        const int run = u >> lcrun, w = u & (crun - 1);
        const uint64_t g = base + __ldg(P.hoff + run) + (uint64_t)(w * kPerCopy);
        cp_async16(chunk + (run << lrun) + w * kPerCopy, psi + g);
    }
    cp_async_commit();
    // 2. coefficients with the phases of the non-local bits folded in; group records.
    //    The source of a term's target differs from it on the group's x, which has
    //    bits outside the CTA's local set only on the cluster bits (t_xnl).
    for (int t = tid; t < nt; t += kThreads) {
        const int tt = t_first + t;
        const double2 c = __ldg(A.t_c + tt);
        const bool neg = __popcll(__ldg(A.t_znl + tt) & (base ^ __ldg(A.t_xnl + tt))) & 1;
        C2 cv;
        cv.x = (R)(neg ? -c.x : c.x);
        cv.y = (R)(neg ? -c.y : c.y);
        sm_c[t] = cv;
        // Z masks in byte-offset units of the chunk (popcount(z << k & s << k) =
        // popcount(z & s)), so sources are addressed without a multiply
        sm_z[t] = __ldg(A.t_zloc + tt) << kEShift;
    }
    for (int g = tid; g < ng; g += kThreads) {
        const int gg = P.g0 + g;
        double ar = 0.0, ai = 0.0;
        for (int tt = A.g_t0[gg]; tt < A.g_tz[gg]; ++tt) {
            const double2 c = __ldg(A.t_c + tt);
            const bool neg = __popcll(__ldg(A.t_znl + tt) & (base ^ __ldg(A.t_xnl + tt))) & 1;
            ar += neg ? -c.x : c.x;
            ai += neg ? -c.y : c.y;
        }
        C2 a;
        a.x = (R)ar;
        a.y = (R)ai;
        sm_a0[g] = a;
        sm_g[g] = make_int4((int)A.g_xloc[gg], A.g_tz[gg] - t_first, A.g_t0[gg + 1] - t_first, (int)A.g_xcl[gg]);
    }
    cp_async_wait<0>();
    __syncthreads();
    // every chunk of the cluster is staged before any CTA reads a peer's
    if (P.cb) cg::this_cluster().sync();
    // 3. targets of the chunk, TPT per thread at a time
    ExpAcc<R> ea;
    const int kLowMask = (1 << lrun) - 1;
    const int g_start = P.diag ? 1 : 0;
    for (int l0 = tid; l0 < nloc; l0 += kThreads * TPT) {
        R accr[TPT], acci[TPT];
        uint32_t tl[TPT];
        uint64_t gidx[TPT];
        C2 prev[TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            tl[j] = (uint32_t)(l0 + j * kThreads);
            gidx[j] = base + __ldg(P.hoff + (tl[j] >> lrun)) + (tl[j] & kLowMask);
            // a later pass adds to the earlier sums: load them now, used after the gather
            if (flags & 8) prev[j] = out[gidx[j]];
        }
        if (P.diag) {
            // x = 0 group: tabulated terms (FP32: hi + lo parts) + its other terms
            const int4 gr = sm_g[0];
            const C2 a0 = sm_a0[0];
            R fr[TPT], fi[TPT], er[TPT], ei[TPT];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                R lr, li;
                const C2 h = ld_tab<R>(A, tl[j], (uint32_t)nloc, lr, li);
                fr[j] = h.x + a0.x;
                fi[j] = h.y + a0.y;
                er[j] = lr;
                ei[j] = li;
            }
            for (int t = gr.y; t < gr.z; ++t) {
                const uint32_t z = sm_z[t];
                const C2 c = sm_c[t];
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const uint32_t par = __popc(z & (tl[j] << kEShift));
                    fr[j] += flip(c.x, par);
                    if (!REALH) fi[j] += flip(c.y, par);
                }
            }
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const C2 amp = chunk[tl[j]];
                const R f_r = fr[j] + er[j];
                if (REALH) {
                    accr[j] = f_r * amp.x;
                    acci[j] = f_r * amp.y;
                } else {
                    const R f_i = fi[j] + ei[j];
                    accr[j] = f_r * amp.x - f_i * amp.y;
                    acci[j] = f_r * amp.y + f_i * amp.x;
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                accr[j] = R(0);
                acci[j] = R(0);
            }
        }
        const char *cb = reinterpret_cast<const char *>(chunk);
        uint32_t tb[TPT];  // byte offsets of the targets in the chunk
#pragma unroll
        for (int j = 0; j < TPT; ++j) tb[j] = tl[j] << kEShift;
        C2 acc2[TPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            acc2[j].x = accr[j];
            acc2[j].y = acci[j];
        }
        // one group's contribution, sources read from `src` (this CTA's chunk, or a
        // peer's through distributed shared memory when x has cluster bits)
        auto group = [&](const char *src, const int4 gr, const C2 a0) {
            const uint32_t xb = (uint32_t)gr.x << kEShift;
            if (REALH && gr.z - gr.y == 1) {
                // one term besides the folded z_loc = 0 ones (a lattice bond: XX + YY)
                const uint32_t z = sm_z[gr.y];
                const R c = sm_c[gr.y].x;
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const uint32_t sb = tb[j] ^ xb;
                    const R f = a0.x + flip(c, __popc(z & sb));
                    fma_real(acc2[j], f, *reinterpret_cast<const C2 *>(src + sb));
                }
                return;
            }
            R fr[TPT], fi[TPT];
            uint32_t sb[TPT];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                sb[j] = tb[j] ^ xb;
                fr[j] = a0.x;
                if (!REALH) fi[j] = a0.y;
            }
            for (int t = gr.y; t < gr.z; ++t) {
                const uint32_t z = sm_z[t];
                const C2 c = sm_c[t];
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const uint32_t par = __popc(z & sb[j]);
                    fr[j] += flip(c.x, par);
                    if (!REALH) fi[j] += flip(c.y, par);
                }
            }
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const C2 amp = *reinterpret_cast<const C2 *>(src + sb[j]);
                if (REALH) {
                    fma_real(acc2[j], fr[j], amp);
                } else {
                    acc2[j].x += fr[j] * amp.x - fi[j] * amp.y;
                    acc2[j].y += fr[j] * amp.y + fi[j] * amp.x;
                }
            }
        };
        for (int g = g_start; g < ng; ++g) {
            const int4 gr = sm_g[g];
            const C2 a0 = sm_a0[g];
            if (gr.w == 0) {
                group(cb, gr, a0);
            } else {
                const char *peer = reinterpret_cast<const char *>(
                    cg::this_cluster().map_shared_rank(chunk, rank ^ (uint32_t)gr.w));
                group(peer, gr, a0);
            }
        }
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            accr[j] = acc2[j].x;
            acci[j] = acc2[j].y;
        }
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            C2 o;
            o.x = accr[j];
            o.y = acci[j];
            if (flags & 8) {
                o.x = prev[j].x + o.x;
                o.y = prev[j].y + o.y;
            }
            out[gidx[j]] = o;
            if (flags & 2) ea.add(chunk[tl[j]], o.x, o.y);
        }
    }
    if (flags & 2) {
        double er = ea.get(0), ei = ea.get(1), h2 = ea.get(2), p2 = ea.get(3);
        __shared__ double red[4][kThreads / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            er += __shfl_down_sync(0xffffffffu, er, o);
            ei += __shfl_down_sync(0xffffffffu, ei, o);
            h2 += __shfl_down_sync(0xffffffffu, h2, o);
            p2 += __shfl_down_sync(0xffffffffu, p2, o);
        }
        const int lane = tid & 31, warp = tid >> 5;
        if (lane == 0) {
            red[0][warp] = er;
            red[1][warp] = ei;
            red[2][warp] = h2;
            red[3][warp] = p2;
        }
        __syncthreads();
        if (tid < 4) {
            double sum = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) sum += red[tid][w];
            partials[(int64_t)blockIdx.x * 4 + tid] = sum;
        }
    }
    // no CTA leaves while a peer may still read its chunk
    if (P.cb) cg::this_cluster().sync();
}

// T(l) = sum of the x = 0 group's terms with z_nl = 0: c (-1)^popc(z_loc & l)
__global__ void k_local_diag_table(int b, int t0, int t1, const uint32_t *zloc, const double2 *c, double2 *tab64,
                                   float2 *tab32) {
    const uint32_t l = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = 1u << b;
    if (l >= n) return;
    double re = 0.0, im = 0.0;
    for (int t = t0; t < t1; ++t) {
        const double2 cc = c[t];
        const bool neg = __popc(zloc[t] & l) & 1;
        re += neg ? -cc.x : cc.x;
        im += neg ? -cc.y : cc.y;
    }
    tab64[l] = make_double2(re, im);
    const float hr = (float)re, hi = (float)im;
    tab32[l] = make_float2(hr, hi);
    tab32[n + l] = make_float2((float)(re - (double)hr), (float)(im - (double)hi));
}

uint32_t compress(uint64_t v, const std::vector<int> &pos) {
    uint32_t r = 0;
    for (size_t j = 0; j < pos.size(); ++j) r |= (uint32_t)((v >> pos[j]) & 1ull) << j;
    return r;
}

}  // namespace

struct LocalPlan {
    int n = 0, npass = 0;
    int run = kLocRun;   // log2 of the contiguous amplitudes of a staged run
    int cb = 0;          // cluster bits: 2^cb CTAs share one window through distributed shared memory
    struct Pass {
        int b = 0, m = 0, nn = 0, g0 = 0, g1 = 0, diag = 0, nt = 0;
        int8_t npos[64] = {};
        int64_t hoff_at = 0;  // offset into hoff
        int64_t nchunk = 0;
    } pass[kLocMaxPass];
    Allocator al;
    uint32_t *g_xloc = nullptr;
    uint32_t *g_xcl = nullptr;
    uint64_t *t_xnl = nullptr;
    int32_t *g_t0 = nullptr, *g_tz = nullptr;
    uint32_t *t_zloc = nullptr;
    uint64_t *t_znl = nullptr;
    double2 *t_c = nullptr;
    uint64_t *hoff = nullptr;
    double2 *dtab64 = nullptr;
    float2 *dtab32 = nullptr;
    bool real = true;         // every coefficient real: the real-coefficient kernel
    void *scratch = nullptr;  // H psi accumulated across passes when the caller wants no output
    int64_t scratch_bytes = 0;
};

void free_local_plan(LocalPlan *lp) {
    if (!lp) return;
    const Allocator &al = lp->al;
    dev_free(al, lp->g_xloc);
    dev_free(al, lp->g_xcl);
    dev_free(al, lp->t_xnl);
    dev_free(al, lp->g_t0);
    dev_free(al, lp->g_tz);
    dev_free(al, lp->t_zloc);
    dev_free(al, lp->t_znl);
    dev_free(al, lp->t_c);
    dev_free(al, lp->hoff);
    dev_free(al, lp->dtab64);
    dev_free(al, lp->dtab32);
    dev_free(al, lp->scratch);
    delete lp;
}

// Passes for the full 2^n space of H, or nullptr when the operator does not fit
// (a mask wider than the local set, too many passes, groups or terms).
namespace {
LocalPlan *build_local_plan_cb(pauli_sum *H, int n, int cb, cudaStream_t st) {
    // window of a pass: kLocBits bits in each CTA plus cb bits across the cluster;
    // with a cluster the staged runs shrink to 16-32 bytes so that the run bits
    // leave room for more bits of X masks
    const int run = cb ? 1 : kLocRun;
    const int wbits = kLocBits + cb;
    if (n < wbits + 1 || n > 40 || H->m == 0 || H->G == 0) return nullptr;
    const int64_t M = H->m, G = H->G;
    if (M > (int64_t)kLocMaxTerms * kLocMaxPass) return nullptr;
    std::vector<uint64_t> z(M), gx(G);
    std::vector<double2> c(M);
    std::vector<int64_t> gs(G + 1);
    PS_CUDA(cudaMemcpyAsync(z.data(), H->z, M * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(c.data(), H->c, M * sizeof(double2), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(gx.data(), H->gx, G * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(gs.data(), H->gstart, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    // groups in the order of their highest bit (x = 0 first); greedy passes
    std::vector<int64_t> order(G);
    for (int64_t g = 0; g < G; ++g) order[g] = g;
    auto top = [](uint64_t v) { return v ? 63 - __builtin_clzll(v) : -1; };
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return top(gx[a]) < top(gx[b]); });
    const uint64_t runmask = (1ull << run) - 1ull;
    std::vector<std::vector<int64_t>> pass_groups;
    std::vector<uint64_t> pass_mask;
    uint64_t cur = runmask;
    std::vector<int64_t> curg;
    for (int64_t g : order) {
        const uint64_t nm = cur | gx[g];
        if (__builtin_popcountll(nm) <= wbits) {
            cur = nm;
            curg.push_back(g);
            continue;
        }
        if (__builtin_popcountll(runmask | gx[g]) > wbits) return nullptr;
        pass_groups.push_back(curg);
        pass_mask.push_back(cur);
        cur = runmask | gx[g];
        curg.assign(1, g);
    }
    pass_groups.push_back(curg);
    pass_mask.push_back(cur);
    if ((int)pass_groups.size() > kLocMaxPass) return nullptr;

    auto lp = new LocalPlan();
    lp->al = H->al;
    lp->n = n;
    lp->run = run;
    lp->cb = cb;
    lp->npass = (int)pass_groups.size();
    std::vector<uint32_t> h_xloc, h_zloc, tab_z, h_xcl;
    std::vector<int32_t> h_t0, h_tz;
    std::vector<uint64_t> h_znl, h_hoff, h_xnl;
    std::vector<double2> h_c, tab_c;
    int tab_b = 0;
    for (int p = 0; p < lp->npass; ++p) {
        uint64_t W = pass_mask[p];
        // fill the window up to wbits with the lowest unused bits
        for (int bit = 0; bit < n && __builtin_popcountll(W) < wbits; ++bit) W |= 1ull << bit;
        // the cluster bits: the cb highest bits of the window above the run bits;
        // L = the bits of one CTA's chunk
        std::vector<int> clpos;
        for (int bit = n - 1; bit >= run && (int)clpos.size() < cb; --bit)
            if ((W >> bit) & 1ull) clpos.insert(clpos.begin(), bit);
        uint64_t clmask = 0;
        for (int bit : clpos) clmask |= 1ull << bit;
        const uint64_t L = W & ~clmask;
        std::vector<int> pos, hpos, npos(clpos);
        for (int bit = 0; bit < n; ++bit) {
            if ((L >> bit) & 1ull) {
                pos.push_back(bit);
                if (bit >= run) hpos.push_back(bit);
            } else if (!((clmask >> bit) & 1ull)) {
                npos.push_back(bit);
            }
        }
        LocalPlan::Pass &P = lp->pass[p];
        P.b = (int)pos.size();
        P.m = (int)hpos.size();
        P.nn = (int)npos.size();
        for (int i = 0; i < P.nn; ++i) P.npos[i] = (int8_t)npos[i];
        P.nchunk = 1ll << P.nn;
        P.hoff_at = (int64_t)h_hoff.size();
        for (uint32_t r = 0; r < (1u << P.m); ++r) {
            uint64_t off = 0;
            for (int j = 0; j < P.m; ++j) off |= (uint64_t)((r >> j) & 1u) << hpos[j];
            h_hoff.push_back(off);
        }
        P.g0 = (int)h_xloc.size();
        const int t_begin = (int)h_c.size();
        for (int64_t g : pass_groups[p]) {
            const bool x0 = gx[g] == 0;  // the x = 0 group sorts first, so it leads pass 0
            h_xloc.push_back(compress(gx[g], pos));
            h_xcl.push_back(compress(gx[g], clpos));
            const uint64_t xnl = gx[g] & ~L;  // only cluster bits: x lies inside the window
            h_t0.push_back((int32_t)h_c.size());
            // terms with z_loc = 0 first (folded per chunk into one constant), then the
            // rest; the x = 0 group's terms with z_nl = 0 go to the table instead
            std::vector<int64_t> zero, rest;
            for (int64_t t = gs[g]; t < gs[g + 1]; ++t) {
                const uint64_t znl = z[t] & ~L;
                const uint32_t zl = compress(z[t], pos);
                if (x0 && znl == 0) {
                    tab_z.push_back(zl);
                    tab_c.push_back(c[t]);
                } else if (zl == 0) {
                    zero.push_back(t);
                } else {
                    rest.push_back(t);
                }
            }
            for (int64_t t : zero) {
                h_zloc.push_back(0);
                h_znl.push_back(z[t] & ~L);
                h_xnl.push_back(xnl);
                h_c.push_back(c[t]);
            }
            h_tz.push_back((int32_t)h_c.size());
            for (int64_t t : rest) {
                h_zloc.push_back(compress(z[t], pos));
                h_znl.push_back(z[t] & ~L);
                h_xnl.push_back(xnl);
                h_c.push_back(c[t]);
            }
            if (x0) {
                P.diag = 1;
                tab_b = P.b;
            }
        }
        P.g1 = (int)h_xloc.size();
        P.nt = (int)h_c.size() - t_begin;
        if (P.g1 - P.g0 > kLocMaxGroups || P.nt > kLocMaxTerms) {
            free_local_plan(lp);
            return nullptr;
        }
    }
    h_t0.push_back((int32_t)h_c.size());
    for (const double2 &cc : h_c) lp->real = lp->real && cc.y == 0.0;
    for (const double2 &cc : tab_c) lp->real = lp->real && cc.y == 0.0;
    auto up = [&](const void *src, size_t bytes) {
        void *d = dev_alloc(lp->al, bytes > 0 ? bytes : 8);
        if (bytes > 0) PS_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
        return d;
    };
    try {
        lp->g_xloc = static_cast<uint32_t *>(up(h_xloc.data(), h_xloc.size() * sizeof(uint32_t)));
        lp->g_xcl = static_cast<uint32_t *>(up(h_xcl.data(), h_xcl.size() * sizeof(uint32_t)));
        lp->t_xnl = static_cast<uint64_t *>(up(h_xnl.data(), h_xnl.size() * sizeof(uint64_t)));
        lp->g_t0 = static_cast<int32_t *>(up(h_t0.data(), h_t0.size() * sizeof(int32_t)));
        lp->g_tz = static_cast<int32_t *>(up(h_tz.data(), h_tz.size() * sizeof(int32_t)));
        lp->t_zloc = static_cast<uint32_t *>(up(h_zloc.data(), h_zloc.size() * sizeof(uint32_t)));
        lp->t_znl = static_cast<uint64_t *>(up(h_znl.data(), h_znl.size() * sizeof(uint64_t)));
        lp->t_c = static_cast<double2 *>(up(h_c.data(), h_c.size() * sizeof(double2)));
        lp->hoff = static_cast<uint64_t *>(up(h_hoff.data(), h_hoff.size() * sizeof(uint64_t)));
        if (tab_b > 0) {
            const int64_t ntab = 1ll << tab_b;
            lp->dtab64 = static_cast<double2 *>(dev_alloc(lp->al, ntab * sizeof(double2)));
            lp->dtab32 = static_cast<float2 *>(dev_alloc(lp->al, 2 * ntab * sizeof(float2)));
            uint32_t *dz = static_cast<uint32_t *>(up(tab_z.data(), tab_z.size() * sizeof(uint32_t)));
            double2 *dc = static_cast<double2 *>(up(tab_c.data(), tab_c.size() * sizeof(double2)));
            k_local_diag_table<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(tab_b, 0, (int)tab_z.size(), dz, dc,
                                                                             lp->dtab64, lp->dtab32);
            PS_CUDA(cudaGetLastError());
            PS_CUDA(cudaStreamSynchronize(st));
            dev_free(lp->al, dz);
            dev_free(lp->al, dc);
        }
        PS_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        free_local_plan(lp);
        throw;
    }
    return lp;
}

}  // namespace

// Passes for the full 2^n space of H, or nullptr when the operator does not fit
// (a mask wider than the window, too many passes, groups or terms).  cluster:
// windows of kLocBits + 3 bits shared by clusters of 8 CTAs (nullptr where the
// device cannot launch clusters).
LocalPlan *build_local_plan(pauli_sum *H, int n, bool cluster, cudaStream_t st) {
    if (!cluster) return build_local_plan_cb(H, n, 0, st);
    int dev = 0, ok = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev));
    if (!ok) return nullptr;
    return build_local_plan_cb(H, n, kLocClusterBits, st);
}

int64_t local_last_chunks(const LocalPlan *lp) { return lp ? lp->pass[lp->npass - 1].nchunk : 0; }
int64_t local_scratch_bytes(const LocalPlan *lp) { return lp ? lp->scratch_bytes : 0; }
int local_passes(const LocalPlan *lp) { return lp ? lp->npass : 0; }

size_t local_smem(const LocalPlan *lp, int p, int dtype) {
    const LocalPlan::Pass &P = lp->pass[p];
    const size_t es = dtype == PAULI_C64 ? 8 : 16;
    return ((size_t)1 << P.b) * es + (size_t)P.nt * (es + 4) + (size_t)(P.g1 - P.g0) * (es + 16) + 16;
}

template <typename R>
static void launch_local_r(LocalPlan *lp, const void *in, void *out, double *partials, int tpt, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    for (int p = 0; p < lp->npass; ++p) {
        const LocalPlan::Pass &Q = lp->pass[p];
        LocalPassDev P;
        P.b = Q.b;
        P.m = Q.m;
        P.nn = Q.nn;
        P.g0 = Q.g0;
        P.g1 = Q.g1;
        P.diag = Q.diag;
        P.run = lp->run;
        P.cb = lp->cb;
        std::memcpy(P.npos, Q.npos, sizeof(P.npos));
        P.hoff = lp->hoff + Q.hoff_at;
        LocalArgs A;
        A.g_xloc = lp->g_xloc;
        A.g_xcl = lp->g_xcl;
        A.t_xnl = lp->t_xnl;
        A.g_t0 = lp->g_t0;
        A.g_tz = lp->g_tz;
        A.t_zloc = lp->t_zloc;
        A.t_znl = lp->t_znl;
        A.t_c = lp->t_c;
        A.dtab64 = lp->dtab64;
        A.dtab32 = lp->dtab32;
        const size_t smem = local_smem(lp, p, sizeof(R) == 4 ? PAULI_C64 : PAULI_C128);
        const bool last = p + 1 == lp->npass;
        const int flags = (p == 0 ? 1 : 8) | ((last && partials) ? 2 : 0);
        auto run = [&](auto kern) {
            smem_optin(reinterpret_cast<const void *>(kern), smem);
            const C2 *pin = static_cast<const C2 *>(in);
            C2 *pout = static_cast<C2 *>(out);
            if (lp->cb == 0) {
                kern<<<(unsigned)Q.nchunk, kThreads, smem, st>>>(P, A, pin, pout, partials, flags);
            } else {
                // clusters of 2^cb consecutive chunks: the same window, one cluster bit value each
                cudaLaunchConfig_t lc = {};
                lc.gridDim = dim3((unsigned)Q.nchunk, 1, 1);
                lc.blockDim = dim3(kThreads, 1, 1);
                lc.dynamicSmemBytes = smem;
                lc.stream = st;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = 1u << lp->cb;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                lc.attrs = at;
                lc.numAttrs = 1;
                PS_CUDA(cudaLaunchKernelEx(&lc, kern, P, A, pin, pout, partials, flags));
            }
            PS_LAUNCH_CHECK();
        };
        if (tpt == 8) {
            if (lp->real) run(k_apply_local<R, true, 8>);
            else run(k_apply_local<R, false, 8>);
        } else {
            if (lp->real) run(k_apply_local<R, true, 4>);
            else run(k_apply_local<R, false, 4>);
        }
    }
}

void launch_local(LocalPlan *lp, const void *in, void *out, int dtype, int64_t dim, double *partials, int tpt,
                  cudaStream_t st) {
    const int64_t bytes = dim * (dtype == PAULI_C64 ? 8 : 16);
    if (!out) {
        if (lp->scratch_bytes < bytes) {
            PS_CUDA(cudaStreamSynchronize(st));
            dev_free(lp->al, lp->scratch);
            lp->scratch = nullptr;
            lp->scratch_bytes = 0;
            lp->scratch = dev_alloc(lp->al, (size_t)bytes);
            lp->scratch_bytes = bytes;
        }
        out = lp->scratch;
    }
    if (dtype == PAULI_C64) launch_local_r<float>(lp, in, out, partials, tpt, st);
    else launch_local_r<double>(lp, in, out, partials, tpt, st);
}

}  // namespace ps
