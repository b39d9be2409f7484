// apply.cu -- dispatch of the gather kernels (apply_kernels.cuh), the fixed-order
// FP64 reduction of pauli_expect and the single-group rotation kernel.
#include <cmath>
#include "apply_kernels.cuh"

namespace ps {
void launch_apply_f32(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out,
                      double *partials, void *split_buf, cudaStream_t st);
void launch_apply_f64(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out,
                      double *partials, void *split_buf, cudaStream_t st);
namespace {

// Fixed-order FP64 reduction of [nparts][4] partials into result[4].
__global__ void __launch_bounds__(1024) k_reduce(const double *partials, int64_t nparts, double *result) {
    __shared__ double sm[4][1024];
    const int t = threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = t; i < nparts; i += 1024)
        for (int k = 0; k < 4; ++k) s[k] += partials[i * 4 + k];
    for (int k = 0; k < 4; ++k) sm[k][t] = s[k];
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < 4; ++k) sm[k][t] += sm[k][t + o];
        __syncthreads();
    }
    if (t < 4) result[t] = sm[t][0];
}

// ---------------------------------------------------------------------------
// rotation by a single-X-mask Hermitian generator
// ---------------------------------------------------------------------------
constexpr int kRotChunk = 256;

template <typename R> __device__ __forceinline__ void sincos_r(R a, R *s, R *c);
template <> __device__ __forceinline__ void sincos_r<float>(float a, float *s, float *c) { sincosf(a, s, c); }
template <> __device__ __forceinline__ void sincos_r<double>(double a, double *s, double *c) { sincos(a, s, c); }

// check_only: record a sector leak in *status and change nothing (the one-time
// leak check that admits a generator to k_rotate_pairs)
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_rotate(SectorView v, Geom geo, int64_t m, uint64_t x, const uint64_t *__restrict__ z,
         const double2 *__restrict__ c, R theta, typename Cx<R>::T *psi, int *status, int check_only) {
    using C2 = typename Cx<R>::T;
    __shared__ uint64_t sm_z[kRotChunk];
    __shared__ C2 sm_c[kRotChunk];
    const RowCtx rc = decode_row<FULL>(v, geo);
    const int tid = threadIdx.x;
    const int64_t col = rc.c0 + tid;
    const bool act = col < rc.dlo;
    const uint32_t xlo = (uint32_t)(x & ((1ull << v.n_lo) - 1ull));
    const uint32_t xhi = (uint32_t)(x >> v.n_lo);
    uint32_t tlo = 0;
    if (act) tlo = FULL ? (uint32_t)col : __ldg(v.list_lo + v.lst_lo_off[rc.blk] + col);
    const uint32_t shi = rc.thi ^ xhi, slo = tlo ^ xlo;
    const uint64_t s = (uint64_t)slo | ((uint64_t)shi << v.n_lo);
    // f_t = sum_k C_k (-1)^popcount(z_k & s)
    R fr = R(0), fi = R(0);
    for (int64_t k0 = 0; k0 < m; k0 += kRotChunk) {
        const int cnt = (m - k0 < kRotChunk) ? (int)(m - k0) : kRotChunk;
        __syncthreads();
        if (tid < cnt) {
            sm_z[tid] = z[k0 + tid];
            const double2 cc = c[k0 + tid];
            C2 cv;
            cv.x = (R)cc.x;
            cv.y = (R)cc.y;
            sm_c[tid] = cv;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const uint32_t par = __popcll(sm_z[k] & s);
            fr += flip(sm_c[k].x, par);
            fi += flip(sm_c[k].y, par);
        }
    }
    if (!act) return;
    int64_t sidx;
    if (FULL) {
        sidx = (int64_t)s;
    } else {
        const int bb = v.blk_of_khi[cls_hi(v, shi)];
        if (bb < 0 || cls_lo(v, slo) != v.klo[bb]) {
            if (fr != R(0) || fi != R(0)) atomicCAS(status, 0, (int)PAULI_ESECTOR);
            return;
        }
        sidx = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb] + (int64_t)__ldg(v.rank_lo + slo);
    }
    if (check_only) return;
    const int64_t tidx = rc.own_base + col;
    if (x == 0) {
        // diagonal generator: psi_t <- exp(-i theta f_t) psi_t (f_t real)
        R sn, cs;
        sincos_r<R>(theta * fr, &sn, &cs);
        const C2 a = psi[tidx];
        C2 o;
        o.x = cs * a.x + sn * a.y;
        o.y = cs * a.y - sn * a.x;
        psi[tidx] = o;
        return;
    }
    if (tidx >= sidx) return;  // the pair is updated by the thread of its lower index
    const R mag = sqrt(fr * fr + fi * fi);
    if (mag == R(0)) return;
    R sn, cs;
    sincos_r<R>(theta * mag, &sn, &cs);
    const R q = sn / mag;
    const C2 a = psi[tidx], b = psi[sidx];
    // w = f b, psi_t' = cs a - i q w ; u = conj(f) a, psi_s' = cs b - i q u
    const R wr = fr * b.x - fi * b.y, wi = fr * b.y + fi * b.x;
    const R ur = fr * a.x + fi * a.y, ui = fr * a.y - fi * a.x;
    C2 na, nb;
    na.x = cs * a.x + q * wi;
    na.y = cs * a.y - q * wr;
    nb.x = cs * b.x + q * ui;
    nb.y = cs * b.y - q * ur;
    psi[tidx] = na;
    psi[sidx] = nb;
}

// Fused step of the adjoint gradient sweep over a product ansatz: each
// lower-index thread of a pair {t, s = t XOR x} adds its part of
// <lam|G|phi> = sum_t conj(lam_t) f_t phi_s (f_s = conj(f_t)) from the input
// values, then rotates both phi and lam by exp(-i theta G).  (The matrix
// element is the same before and after, since G commutes with its own
// exponential.)  Fixed grid; block b handles work units b, b + gridDim.x, ...
// and writes its FP64 sum to partials[4b..4b+1], so the result is
// reproducible.
template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_rotate_adj(SectorView v, Geom geo, int64_t nwork, int64_t m, uint64_t x, const uint64_t *__restrict__ z,
             const double2 *__restrict__ c, R theta, typename Cx<R>::T *phi, typename Cx<R>::T *lam,
             double *partials, int *status) {
    using C2 = typename Cx<R>::T;
    __shared__ uint64_t sm_z[kRotChunk];
    __shared__ C2 sm_c[kRotChunk];
    __shared__ double red[2][kThreads / 32];
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
        for (int64_t k0 = 0; k0 < m; k0 += kRotChunk) {
            const int cnt = (m - k0 < kRotChunk) ? (int)(m - k0) : kRotChunk;
            __syncthreads();
            if (tid < cnt) {
                sm_z[tid] = z[k0 + tid];
                const double2 cc = c[k0 + tid];
                C2 cv;
                cv.x = (R)cc.x;
                cv.y = (R)cc.y;
                sm_c[tid] = cv;
            }
            __syncthreads();
            for (int k = 0; k < cnt; ++k) {
                const uint32_t par = __popcll(sm_z[k] & s);
                fr += flip(sm_c[k].x, par);
                fi += flip(sm_c[k].y, par);
            }
        }
        if (!act) continue;
        int64_t sidx;
        if (FULL) {
            sidx = (int64_t)s;
        } else {
            const int bb = v.blk_of_khi[cls_hi(v, shi)];
            if (bb < 0 || cls_lo(v, slo) != v.klo[bb]) {
                if (fr != R(0) || fi != R(0)) atomicCAS(status, 0, (int)PAULI_ESECTOR);
                continue;
            }
            sidx = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb] + (int64_t)__ldg(v.rank_lo + slo);
        }
        const int64_t tidx = rc.own_base + col;
        if (x == 0) {
            const C2 a = phi[tidx], la = lam[tidx];
            C2 fa;
            fa.x = fr * a.x;
            fa.y = fr * a.y;
            dot.add(la, fa);
            R sn, cs;
            sincos_r<R>(theta * fr, &sn, &cs);
            C2 o, lo;
            o.x = cs * a.x + sn * a.y;
            o.y = cs * a.y - sn * a.x;
            lo.x = cs * la.x + sn * la.y;
            lo.y = cs * la.y - sn * la.x;
            phi[tidx] = o;
            lam[tidx] = lo;
            continue;
        }
        if (tidx >= sidx) continue;
        const R mag = sqrt(fr * fr + fi * fi);
        if (mag == R(0)) continue;
        const C2 a = phi[tidx], b = phi[sidx], la = lam[tidx], lb = lam[sidx];
        // conj(la) f b + conj(lb) conj(f) a
        {
            C2 fb, fa;
            fb.x = fr * b.x - fi * b.y;
            fb.y = fr * b.y + fi * b.x;
            fa.x = fr * a.x + fi * a.y;
            fa.y = fr * a.y - fi * a.x;
            dot.add(la, fb);
            dot.add(lb, fa);
        }
        R sn, cs;
        sincos_r<R>(theta * mag, &sn, &cs);
        const R q = sn / mag;
        auto rot = [&](const C2 &u, const C2 &w, C2 &nu, C2 &nw) {
            const R wr = fr * w.x - fi * w.y, wi = fr * w.y + fi * w.x;
            const R ur = fr * u.x + fi * u.y, ui = fr * u.y - fi * u.x;
            nu.x = cs * u.x + q * wi;
            nu.y = cs * u.y - q * wr;
            nw.x = cs * w.x + q * ui;
            nw.y = cs * w.y - q * ur;
        };
        C2 na, nb, nla, nlb;
        rot(a, b, na, nb);
        rot(la, lb, nla, nlb);
        phi[tidx] = na;
        phi[sidx] = nb;
        lam[tidx] = nla;
        lam[sidx] = nlb;
    }
    double mr = dot.get_re(), mi = dot.get_im();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mr += __shfl_down_sync(0xffffffffu, mr, o);
        mi += __shfl_down_sync(0xffffffffu, mi, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = mr;
        red[1][tid >> 5] = mi;
    }
    __syncthreads();
    if (tid < 2) {
        double acc = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) acc += red[tid][w];
        partials[(int64_t)blockIdx.x * 4 + tid] = acc;
    }
}

// The same rotation (ADJ: the adjoint step of k_rotate_adj) over the listed
// pairs only (RotPairs): no work for targets whose partner leaves the block, and
// each pair is visited once.  Fixed grid, block-strided over pair ids.
// Angles of one rotation per active pattern (ActivePatterns), from the host:
// f(s) = (-1)^{z_o . s} F_k for a target with t & S = pat[k], and
// cos(theta |F_k|), sin(theta |F_k|) / |F_k| once per launch instead of per pair.
template <typename R>
struct RotAngles {
    uint64_t S, zo;
    uint64_t pat[kActMax];
    R fr[kActMax], fi[kActMax];
    R cs[kActMax], q[kActMax];
    int np;  // 0: every pair sums its terms and takes its own sin / cos
};

template <typename R, bool ADJ>
__global__ void __launch_bounds__(kThreads)
k_rotate_pairs(int64_t npairs, int64_t nlo, const uint32_t *__restrict__ tab, int64_t nhi, int n_lo, int64_t off,
               int64_t dlo, int64_t m, uint64_t x, const uint64_t *__restrict__ z, const double2 *__restrict__ c,
               R theta, RotAngles<R> ra, typename Cx<R>::T *phi, typename Cx<R>::T *lam, double *partials) {
    using C2 = typename Cx<R>::T;
    __shared__ uint64_t sm_z[kRotPairTerms];
    __shared__ C2 sm_c[kRotPairTerms];
    __shared__ double red[2][kThreads / 32];
    const int tid = threadIdx.x;
    for (int k = tid; k < m; k += kThreads) {
        sm_z[k] = z[k];
        const double2 cc = c[k];
        C2 cv;
        cv.x = (R)cc.x;
        cv.y = (R)cc.y;
        sm_c[k] = cv;
    }
    __syncthreads();
    const uint32_t *pat_lo = tab, *rt_lo = tab + nlo, *rs_lo = tab + 2 * nlo;
    const uint32_t *pat_hi = tab + 3 * nlo, *rt_hi = pat_hi + nhi, *rs_hi = pat_hi + 2 * nhi;
    DotAcc<R> dot;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + tid; i < npairs; i += (int64_t)gridDim.x * kThreads) {
        const int64_t h = i / nlo, l = i - h * nlo;
        const uint64_t t = ((uint64_t)__ldg(pat_hi + h) << n_lo) | (uint64_t)__ldg(pat_lo + l);
        const uint64_t s = t ^ x;
        R fr = R(0), fi = R(0), cs, q;
        if (ra.np != 0) {
            const uint64_t tm = t & ra.S;
            int kk = -1;
#pragma unroll
            for (int k = 0; k < kActMax; ++k)
                if (k < ra.np && tm == ra.pat[k]) kk = k;
            if (kk < 0) continue;  // f = 0: the pair does not rotate
            const uint32_t par = __popcll(ra.zo & s);
            fr = flip(ra.fr[kk], par);
            fi = flip(ra.fi[kk], par);
            cs = ra.cs[kk];
            q = ra.q[kk];
        } else {
            for (int k = 0; k < m; ++k) {
                const uint32_t par = __popcll(sm_z[k] & s);
                fr += flip(sm_c[k].x, par);
                fi += flip(sm_c[k].y, par);
            }
            const R mag = sqrt(fr * fr + fi * fi);
            if (mag == R(0)) continue;
            R sn;
            sincos_r<R>(theta * mag, &sn, &cs);
            q = sn / mag;
        }
        const int64_t it = off + (int64_t)__ldg(rt_hi + h) * dlo + __ldg(rt_lo + l);
        const int64_t is = off + (int64_t)__ldg(rs_hi + h) * dlo + __ldg(rs_lo + l);
        auto rot = [&](const C2 &u, const C2 &w, C2 &nu, C2 &nw) {
            const R wr = fr * w.x - fi * w.y, wi = fr * w.y + fi * w.x;
            const R ur = fr * u.x + fi * u.y, ui = fr * u.y - fi * u.x;
            nu.x = cs * u.x + q * wi;
            nu.y = cs * u.y - q * wr;
            nw.x = cs * w.x + q * ui;
            nw.y = cs * w.y - q * ur;
        };
        const C2 a = phi[it], b = phi[is];
        C2 na, nb;
        rot(a, b, na, nb);
        phi[it] = na;
        phi[is] = nb;
        if (ADJ) {
            const C2 la = lam[it], lb = lam[is];
            // conj(la) f b + conj(lb) conj(f) a, from the input values
            C2 fb, fa;
            fb.x = fr * b.x - fi * b.y;
            fb.y = fr * b.y + fi * b.x;
            fa.x = fr * a.x + fi * a.y;
            fa.y = fr * a.y - fi * a.x;
            dot.add(la, fb);
            dot.add(lb, fa);
            C2 nla, nlb;
            rot(la, lb, nla, nlb);
            lam[it] = nla;
            lam[is] = nlb;
        }
    }
    if (ADJ) {
        double mr = dot.get_re(), mi = dot.get_im();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mr += __shfl_down_sync(0xffffffffu, mr, o);
            mi += __shfl_down_sync(0xffffffffu, mi, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = mr;
            red[1][tid >> 5] = mi;
        }
        __syncthreads();
        if (tid < 2) {
            double acc = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) acc += red[tid][w];
            partials[(int64_t)blockIdx.x * 4 + tid] = acc;
        }
    }
}

}  // namespace

// 227 KB of shared memory per block on sm_103a, less room for the kernel's static arrays
constexpr size_t kMaxDynSmem = 226 * 1024;

const LaunchChoice *find_tuned(const Plan &p, const SectorView &v, int dtype) {
    for (const TunedEntry &t : p.tuned)
        if (t.dim == v.dim && t.nblk == v.nblk && t.dtype == dtype) return &t.choice;
    return nullptr;
}

// Launch shape of one apply.  Each field is resolved from, in order: the
// forced choice (the autotuner's candidate), the plan's tuned entry for this
// sector and dtype (pauli_set_launch_config / pauli_tune), the heuristics.
ApplyCfg apply_config(const Plan &p, const SectorView &v, int dtype, bool allow_split, const LaunchChoice *force) {
    ApplyCfg c;
    LaunchChoice ch;
    if (force) ch = *force;
    else if (const LaunchChoice *t = find_tuned(p, v, dtype)) ch = *t;
    auto buf_bytes = [&](int cap) {
        return dtype == PAULI_C64 ? Smem<float>::buf_bytes(cap) : Smem<double>::buf_bytes(cap);
    };
    int64_t mx = 0;
    for (int b = 0; b < v.nblk; ++b) mx = std::max(mx, v.dlo[b]);
    // rows staged by bit pattern need 2^n_lo slots; a single block can instead
    // be staged densely by rank (D_lo slots) plus a rank table
    const bool single = v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1;
    const size_t bb_pattern = buf_bytes(1 << v.n_lo);
    const bool rank_ok = single && v.n_lo <= (v.irr ? 14 : 16);
    const int dflt_ranked = (single && bb_pattern > kMaxDynSmem) ? 1 : 0;
    c.ranked = rank_ok && (ch.ranked >= 0 ? ch.ranked != 0 : dflt_ranked != 0);
    const size_t bb = c.ranked ? buf_bytes(ranked_rowcap(v.dlo[0])) : bb_pattern;
    const size_t extra = c.ranked ? rank_table_bytes(v.n_lo) : 0;
    // measured on the 24-qubit molecule (D_lo = 924): 4 columns per thread and a
    // single staged row (more resident CTAs) beat finer tiles and double buffering
    // rank-staged rows wider than ~100 KB leave one or two CTAs per SM: 8 columns per
    // thread then give each thread more independent gathers to overlap
    const bool wide_ranked = c.ranked && bb + extra > 100 * 1024 && mx >= 6 * kThreads;
    int tpt = ch.tpt ? ch.tpt : (wide_ranked ? 8 : mx >= 3 * kThreads ? 4 : (mx >= 3 * kThreads / 2 ? 2 : 1));
    if (tpt == 8 && !c.ranked) tpt = 4;
    if (tpt != 1 && tpt != 2 && tpt != 4 && tpt != 8) tpt = 1;
    int nbuf = ch.nbuf ? ch.nbuf : 1;
    if (nbuf != 1 && nbuf != 2) nbuf = 1;
    if (tpt == 8) nbuf = 1;  // 8 columns per thread exist for one staged row only
    if (nbuf * bb + extra > kMaxDynSmem) nbuf = 1;
    c.tpt = tpt;
    c.nbuf = nbuf;
    c.smem = nbuf * bb + extra;
    c.base_nct = make_geom(v, tpt * kThreads).cta_off[v.nblk];
    // SVD-factorised phases (installed or tuned; the plan must have been built for
    // this sector's low half): one staged row per piece of groups sharing x_hi
    if (ch.direct == 4 && svd_plan_fits(p.svd, v)) {
        int t = ch.tpt == 2 || ch.tpt == 4 ? ch.tpt : 1;
        c.svd = true;
        c.ranked = true;
        c.list = false;
        c.tpt = t;
        c.nbuf = 1;
        c.smem = svd_smem(v, dtype);
        c.base_nct = make_geom(v, t * kThreads).cta_off[v.nblk];
        c.nsplit = 1;
        c.split_p0.assign(2, 0);
        c.split_p0[1] = (int32_t)p.P;
        c.nct = c.base_nct;
        c.combine_nct = 0;
        return c;
    }
    // full space with a local-pass plan (lattice operators, 2^21 amplitudes or more):
    // chunks staged in shared memory, one pass per local bit set
    if (v.kind == PAULI_SECTOR_FULL && (p.local || p.local_cl)) {
        const int dflt_local = v.n >= 21 ? 1 : 0;
        if (ch.direct >= 0 ? ch.direct == 2 : dflt_local != 0) {
            // clustered windows only where installed (ranked = 1) or where the plain
            // chunks do not fit: they move fewer bytes (two passes instead of three at
            // 26-30 sites) but the cluster barriers leave the issue-bound gather slower
            // (30 sites: 35.8 ms against 23.0 ms)
            bool cl;
            if (ch.direct == 2 && ch.ranked >= 0) cl = ch.ranked == 1 ? p.local_cl != nullptr : p.local == nullptr;
            else cl = p.local == nullptr;
            c.local = true;
            c.local_cl = cl;
            c.ranked = cl;
            c.tpt = ch.tpt == 8 ? 8 : 4;  // targets per thread of the pass kernel
            c.direct = false;
            c.smem = 0;
            c.nbuf = 1;
            c.nsplit = 1;
            c.split_p0.assign(2, 0);
            c.split_p0[1] = (int32_t)p.P;
            c.nct = local_last_chunks(cl ? p.local_cl : p.local);
            c.combine_nct = 0;
            return c;
        }
    }
    // a single block with a low half of at most kListMaxLo qubits: gather over
    // the lists of valid (target, source) pairs, one CTA per row (list.cu)
    const std::vector<int64_t> *cumw = &p.h_pc_cumw;
    const ListTab *lt = single ? find_lists(p, v.klo[0]) : nullptr;
    bool use_list = false;
    if (lt) {
        const int dflt_list = (dtype == PAULI_C128 && v.dlo[0] >= 384) ? 1 : 0;
        use_list = ch.direct >= 0 ? ch.direct == 3 : dflt_list != 0;
    }
    if (use_list) {
        c.list = true;
        c.ranked = false;
        c.tpt = 1;
        c.nbuf = 1;
        c.smem = list_smem(dtype, v.dlo[0]);
        c.base_nct = v.dlo[0] > 0 ? v.dhi[0] : 0;
        cumw = &lt->h_pc_cumw;
    }
    // small operators (lattice models): the whole folded plan fits in shared
    // memory and rows have few pieces, so gather straight from global memory
    const bool fits = p.I <= kDirectItems && p.S <= kDirectSegs;
    const int dflt_direct = fits ? 1 : 0;
    c.direct = !use_list && fits && (ch.direct >= 0 ? ch.direct == 1 : dflt_direct != 0);
    if (c.direct) {
        // the direct gather stages nothing and has 1, 2 or 4 columns per thread
        c.ranked = false;
        if (c.tpt == 8) c.tpt = 4;
        c.base_nct = make_geom(v, c.tpt * kThreads).cta_off[v.nblk];
        c.smem = 0;
        c.nbuf = 1;
        c.nsplit = 1;
        c.split_p0.assign(2, 0);
        c.split_p0[1] = (int32_t)p.P;
        c.nct = c.base_nct;
        c.combine_nct = 0;
        return c;
    }
    // Too few rows for the GPU: split each row's pieces into nsplit balanced
    // ranges (by the plan's per-piece work estimate) so that a launch has about
    // sixteen waves of CTAs (finer units even out the uneven pieces; measured on
    // the 24-qubit molecule: 3.78 ms at four waves, 3.55 ms at sixteen);
    // k_combine adds the partial vectors in a fixed order.
    int nsplit = 1;
    if (allow_split && c.base_nct > 0 && p.P > 1) {
        const int per_sm = std::max<int>(1, std::min<int>(2048 / kThreads, (int)((228 * 1024) / (c.smem + 2048))));
        const int64_t slots = (int64_t)num_sms() * per_sm;
        if (c.base_nct < 16 * slots) nsplit = (int)((16 * slots + c.base_nct - 1) / c.base_nct);
        if (ch.nsplit) nsplit = ch.nsplit;
        nsplit = std::max(1, std::min<int>({nsplit, kMaxSplit, (int)std::max<int64_t>(1, p.P / 8)}));
    }
    c.nsplit = nsplit;
    c.split_p0.assign(nsplit + 1, 0);
    const int64_t W = cumw->empty() ? 0 : cumw->back();
    for (int k = 1; k < nsplit; ++k) {
        const int64_t target = W * k / nsplit;
        const int32_t q = (int32_t)(std::lower_bound(cumw->begin(), cumw->end(), target) - cumw->begin());
        c.split_p0[k] = std::max(c.split_p0[k - 1], std::min<int32_t>(q, (int32_t)p.P));
    }
    c.split_p0[nsplit] = (int32_t)p.P;
    c.nct = c.base_nct * nsplit;
    c.combine_nct = nsplit > 1 ? (v.dim + kThreads - 1) / kThreads : 0;
    return c;
}

int64_t apply_num_ctas(const Plan &p, const SectorView &v, int dtype, bool allow_split, const LaunchChoice *force) {
    const ApplyCfg c = apply_config(p, v, dtype, allow_split, force);
    if (c.local) return c.nct;  // the last pass writes the partials
    return c.nsplit > 1 ? c.combine_nct : c.base_nct;
}

int64_t apply_split_elems(const Plan &p, const SectorView &v, int dtype, const LaunchChoice *force) {
    const ApplyCfg c = apply_config(p, v, dtype, true, force);
    return c.nsplit > 1 ? (int64_t)c.nsplit * v.dim : 0;
}

void launch_apply(pauli_sum *H, const Plan &p, const SectorView &v, const void *psi_in, void *psi_out,
                  int dtype, double *partials, cudaStream_t st, bool allow_split, const LaunchChoice *force) {
    (void)H;
    const ApplyCfg cfg = apply_config(p, v, dtype, allow_split, force);
    if (cfg.nct == 0) return;
    PS_CHECK(cfg.nct < (1ll << 31), PAULI_EUNSUPPORTED, "apply: too many thread blocks");
    if (cfg.local) {
        launch_local(cfg.local_cl ? p.local_cl : p.local, psi_in, psi_out, dtype, v.dim, partials, cfg.tpt, st);
        return;
    }
    PS_CHECK(cfg.smem <= kMaxDynSmem, PAULI_EUNSUPPORTED,
             "apply: the low half of the sector split is too wide for shared-memory staging");
    void *split_buf = nullptr;
    if (cfg.nsplit > 1) {
        const int64_t need = (int64_t)cfg.nsplit * v.dim * (dtype == PAULI_C64 ? 8 : 16);
        PS_CHECK(p.split_buf != nullptr && p.split_cap >= need, PAULI_EINVAL,
                 "apply: the plan's split buffer is missing (internal)");
        split_buf = p.split_buf;
    }
    if (cfg.list) {
        launch_list(cfg, p, v, psi_in, psi_out, dtype, partials, split_buf, st);
        return;
    }
    if (cfg.svd) {
        launch_svd(cfg, p, v, psi_in, psi_out, dtype, partials, st);
        return;
    }
    if (dtype == PAULI_C64) launch_apply_f32(cfg, p, v, psi_in, psi_out, partials, split_buf, st);
    else launch_apply_f64(cfg, p, v, psi_in, psi_out, partials, split_buf, st);
}

void launch_reduce(const double *partials, int64_t nparts, double *result, cudaStream_t st) {
    k_reduce<<<1, 1024, 0, st>>>(partials, nparts, result);
    PS_LAUNCH_CHECK();
}
// X mask of a single-group operator, read back from the device once
uint64_t group_mask0(pauli_sum *G) {
    if (!G->gx0_known) {
        uint64_t x = 0;
        if (G->G == 1) PS_CUDA(cudaMemcpy(&x, G->gx, sizeof(uint64_t), cudaMemcpyDeviceToHost));
        G->gx0_host = x;
        G->gx0_known = true;
    }
    return G->gx0_host;
}

// colex rank of a string among the strings of the same popcount: sum over its
// set bits p_0 < p_1 < ... of C(p_j, j + 1)
static uint32_t colex_rank(uint32_t b) {
    uint64_t r = 0;
    int j = 0;
    while (b) {
        const int p = __builtin_ctz(b);
        uint64_t cnk = 0;
        if (p >= j + 1) {
            cnk = 1;
            for (int i = 0; i < j + 1; ++i) cnk = cnk * (uint64_t)(p - i) / (uint64_t)(i + 1);
        }
        r += cnk;
        ++j;
        b &= b - 1;
    }
    return (uint32_t)r;
}

// The strings of `bits` bits with popcount k that have exactly half of xm's bits
// set (and bit `need`, if need >= 0), ascending, with their ranks and the ranks
// of b ^ xm.
static void half_pairs(int bits, int k, uint32_t xm, int need, std::vector<uint32_t> &pat,
                       std::vector<uint32_t> &rt, std::vector<uint32_t> &rs) {
    const int a = __builtin_popcount(xm);
    if (k < 0 || k > bits) return;
    if (k == 0) {
        if (a == 0 && need < 0) {
            pat.push_back(0);
            rt.push_back(0);
            rs.push_back(0);
        }
        return;
    }
    // Gosper's rule: the k-subsets of `bits` bits in increasing order (= colex rank order)
    uint64_t b = (1ull << k) - 1ull;
    const uint64_t lim = 1ull << bits;
    uint32_t rank = 0;
    while (b < lim) {
        const uint32_t bb = (uint32_t)b;
        if (2 * __builtin_popcount(bb & xm) == a && (need < 0 || ((bb >> need) & 1u))) {
            pat.push_back(bb);
            rt.push_back(rank);
            rs.push_back(colex_rank(bb ^ xm));
        }
        ++rank;
        const uint64_t cbit = b & (~b + 1ull), r = b + cbit;
        b = (((r ^ b) >> 2) / cbit) | r;
    }
}

// One-time check: does G move amplitude out of the sector?  (k_rotate in
// check-only mode; the answer is read back, so the call synchronises st once.)
static bool rotation_leaks(pauli_sum *G, const SectorView &v, uint64_t x, cudaStream_t st) {
    if (!G->leak_flag) G->leak_flag = static_cast<int *>(dev_alloc(G->al, sizeof(int)));
    PS_CUDA(cudaMemsetAsync(G->leak_flag, 0, sizeof(int), st));
    const Geom geo = make_geom(v, kThreads);
    const int64_t nct = geo.cta_off[v.nblk];
    if (nct > 0) {
        PS_CHECK(nct < (1ll << 31), PAULI_EUNSUPPORTED, "rotate: too many thread blocks");
        k_rotate<double, false><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, 0.0, nullptr,
                                                                    G->leak_flag, 1);
        PS_LAUNCH_CHECK();
    }
    int flag = 0;
    PS_CUDA(cudaMemcpyAsync(&flag, G->leak_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    return flag != 0;
}

// Pair tables of (G, sector) for k_rotate_pairs, built on first use and kept in G
// (the last kRotPairsCache sectors); nullptr where the per-target kernel applies:
// full space, several blocks, x = 0, more than kRotPairTerms terms, or a generator
// that leaks out of the sector (its leaks are then recorded on every call).
const RotPairs *rotation_pairs(pauli_sum *G, const pauli_sector *sec, uint64_t x, cudaStream_t st) {
    const SectorView &v = sec->v;
    if (v.kind != PAULI_SECTOR_BLOCKS || v.nblk != 1 || v.irr || x == 0 || G->m > kRotPairTerms) return nullptr;
    for (int i = 0; i < G->nrot; ++i)
        if (G->rot[i].sector_uid == sec->uid) return G->rot[i].leaks ? nullptr : &G->rot[i];
    RotPairs rp;
    rp.sector_uid = sec->uid;
    rp.leaks = rotation_leaks(G, v, x, st) ? 1 : 0;
    if (!rp.leaks) {
        {
            std::vector<uint64_t> hz(G->m);
            std::vector<double2> hc(G->m);
            PS_CUDA(cudaMemcpyAsync(hz.data(), G->z, G->m * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
            PS_CUDA(cudaMemcpyAsync(hc.data(), G->c, G->m * sizeof(double2), cudaMemcpyDeviceToHost, st));
            PS_CUDA(cudaStreamSynchronize(st));
            rp.act = find_active_patterns(x, hz.data(), hc.data(), G->m);
        }
        const uint32_t lomask = (uint32_t)((1ull << v.n_lo) - 1ull);
        const uint32_t xlo = (uint32_t)(x & lomask), xhi = (uint32_t)(x >> v.n_lo);
        const int b0 = __builtin_ctzll(x);
        std::vector<uint32_t> plo, rtlo, rslo, phi, rthi, rshi;
        half_pairs(v.n_lo, v.klo[0], xlo, b0 < v.n_lo ? b0 : -1, plo, rtlo, rslo);
        half_pairs(v.n_hi, v.khi[0], xhi, b0 >= v.n_lo ? b0 - v.n_lo : -1, phi, rthi, rshi);
        rp.nlo = (int64_t)plo.size();
        rp.nhi = (int64_t)phi.size();
        std::vector<uint32_t> tab;
        tab.reserve(3 * (rp.nlo + rp.nhi));
        for (auto *vv : {&plo, &rtlo, &rslo, &phi, &rthi, &rshi}) tab.insert(tab.end(), vv->begin(), vv->end());
        if (!tab.empty()) {
            rp.tab = static_cast<uint32_t *>(dev_alloc(G->al, tab.size() * sizeof(uint32_t)));
            PS_CUDA(cudaMemcpyAsync(rp.tab, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
            PS_CUDA(cudaStreamSynchronize(st));
        }
    }
    if (G->nrot == kRotPairsCache) {
        dev_free(G->al, G->rot[0].tab);
        for (int i = 1; i < kRotPairsCache; ++i) G->rot[i - 1] = G->rot[i];
        --G->nrot;
    }
    G->rot[G->nrot++] = rp;
    const RotPairs &r = G->rot[G->nrot - 1];
    return r.leaks ? nullptr : &r;
}

template <typename R, bool ADJ>
static void launch_pairs(const RotPairs &rp, pauli_sum *G, const SectorView &v, uint64_t x, double theta, void *phi,
                         void *lam, double *partials, unsigned grid, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    RotAngles<R> ra;
    const ActivePatterns &ap = rp.act;
    ra.S = ap.S;
    ra.zo = ap.zo;
    ra.np = ap.np;
    for (int k = 0; k < kActMax; ++k) {
        const double mag = std::hypot(ap.F[k].x, ap.F[k].y);
        ra.pat[k] = ap.pat[k];
        ra.fr[k] = (R)ap.F[k].x;
        ra.fi[k] = (R)ap.F[k].y;
        ra.cs[k] = (R)std::cos(theta * mag);
        ra.q[k] = (R)(mag > 0.0 ? std::sin(theta * mag) / mag : 0.0);
    }
    k_rotate_pairs<R, ADJ><<<grid, kThreads, 0, st>>>(rp.nlo * rp.nhi, rp.nlo > 0 ? rp.nlo : 1, rp.tab, rp.nhi,
                                                     v.n_lo, v.off[0], v.dlo[0], G->m, x, G->z, G->c, (R)theta, ra,
                                                     static_cast<C2 *>(phi), static_cast<C2 *>(lam), partials);
    PS_LAUNCH_CHECK();
}

void launch_rotate_adjoint(pauli_sum *G, const pauli_sector *sec, double theta, void *phi, void *lam, int dtype,
                           double *result, cudaStream_t st) {
    const SectorView &v = sec->v;
    const uint64_t x = group_mask0(G);
    if (const RotPairs *rp = rotation_pairs(G, sec, x, st)) {
        DotScratch &d = dot_scratch();
        const int64_t np = rp->nlo * rp->nhi;
        const int64_t need = (np + kThreads - 1) / kThreads;
        const unsigned grid = (unsigned)(need < d.blocks ? (need > 0 ? need : 1) : d.blocks);
        if (dtype == PAULI_C64) launch_pairs<float, true>(*rp, G, v, x, theta, phi, lam, d.partials, grid, st);
        else launch_pairs<double, true>(*rp, G, v, x, theta, phi, lam, d.partials, grid, st);
        launch_reduce2(d.partials, grid, result, st);
        return;
    }

    const Geom geo = make_geom(v, kThreads);
    const int64_t nwork = geo.cta_off[v.nblk];
    DotScratch &d = dot_scratch();
    const unsigned grid = (unsigned)(nwork < d.blocks ? (nwork > 0 ? nwork : 1) : d.blocks);
    const bool full = v.kind == PAULI_SECTOR_FULL;
    if (dtype == PAULI_C64) {
        auto *a = static_cast<float2 *>(phi);
        auto *b = static_cast<float2 *>(lam);
        if (full) k_rotate_adj<float, true><<<grid, kThreads, 0, st>>>(v, geo, nwork, G->m, x, G->z, G->c, (float)theta, a, b, d.partials, G->status);
        else k_rotate_adj<float, false><<<grid, kThreads, 0, st>>>(v, geo, nwork, G->m, x, G->z, G->c, (float)theta, a, b, d.partials, G->status);
    } else {
        auto *a = static_cast<double2 *>(phi);
        auto *b = static_cast<double2 *>(lam);
        if (full) k_rotate_adj<double, true><<<grid, kThreads, 0, st>>>(v, geo, nwork, G->m, x, G->z, G->c, theta, a, b, d.partials, G->status);
        else k_rotate_adj<double, false><<<grid, kThreads, 0, st>>>(v, geo, nwork, G->m, x, G->z, G->c, theta, a, b, d.partials, G->status);
    }
    PS_LAUNCH_CHECK();
    launch_reduce2(d.partials, grid, result, st);
}

void launch_rotate(pauli_sum *G, const pauli_sector *sec, double theta, void *psi, int dtype,
                   cudaStream_t st) {
    const SectorView &v = sec->v;
    const uint64_t x = group_mask0(G);
    if (const RotPairs *rp = rotation_pairs(G, sec, x, st)) {
        const int64_t np = rp->nlo * rp->nhi;
        if (np == 0) return;
        const int blocks = num_sms() * 8;
        const int64_t need = (np + kThreads - 1) / kThreads;
        const unsigned grid = (unsigned)(need < blocks ? need : blocks);
        if (dtype == PAULI_C64) launch_pairs<float, false>(*rp, G, v, x, theta, psi, nullptr, nullptr, grid, st);
        else launch_pairs<double, false>(*rp, G, v, x, theta, psi, nullptr, nullptr, grid, st);
        return;
    }
    const Geom geo = make_geom(v, kThreads);
    const int64_t nct = geo.cta_off[v.nblk];
    if (nct == 0) return;
    PS_CHECK(nct < (1ll << 31), PAULI_EUNSUPPORTED, "rotate: too many thread blocks");
    const bool full = v.kind == PAULI_SECTOR_FULL;
    if (dtype == PAULI_C64) {
        if (full) k_rotate<float, true><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, (float)theta, static_cast<float2 *>(psi), G->status, 0);
        else k_rotate<float, false><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, (float)theta, static_cast<float2 *>(psi), G->status, 0);
    } else {
        if (full) k_rotate<double, true><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, theta, static_cast<double2 *>(psi), G->status, 0);
        else k_rotate<double, false><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, theta, static_cast<double2 *>(psi), G->status, 0);
    }
    PS_LAUNCH_CHECK();
}

}  // namespace ps
