// apply.cu -- operator-state kernels of the gather family (Sec. 2.4):
//   k_apply   (H psi)_t  = sum_g psi[t ^ x_g] f_g(t),
//             f_g(t)     = sum_{k in g} C_k (-1)^popcount(z_k & (t ^ x_g))
//             (eq. reverse_sum / eq. sreverse_sum), with the expectation
//             value <psi|H|psi> and ||H psi||^2 reduced in FP64 (eq. vqe_energy);
//   k_rotate  psi <- exp(-i theta G) psi for a single-X-mask Hermitian G.
//
// Work decomposition.  A target t = (t_hi, t_lo) lives in a row (its high
// half: the beta string of a molecule) and a column (its low half: the alpha
// string).  One CTA owns one row and a tile of its columns; its threads own
// columns, so every output element is written by exactly one thread and no
// atomics are needed (the paper's race-free target-driven summation).
//
// Because the row is fixed inside a CTA, the high half of every phase
//   (-1)^popcount(z_hi & s_hi),  s_hi = t_hi ^ x_hi(g)
// is the same for all of the CTA's targets (the alpha/beta factorisation of
// eq. sreverse_sum).  The plan stores each group's terms sorted by (z_lo, z_hi)
// so that terms sharing z_lo form a segment; the CTA first folds the high-half
// phases into one coefficient per segment,
//   a_seg = sum_{k in seg} C_k (-1)^popcount(z_hi,k & s_hi),
// in shared memory, and the per-target loop is then
//   f_g(t) = sum_{seg in g} a_seg (-1)^popcount(z_lo,seg & s_lo),
// popcount parity applied as a sign-bit flip.  The source index is
//   off_r' + rank_hi(s_hi) D_lo^r' + rank_lo(s_lo),
// the first two terms per (row, group) in shared memory, rank_lo from a
// table filled with the binomial colex ranking.
#include <algorithm>

#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kThreads = 256;

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ float flip(float a, uint32_t parity_word) {
    return __int_as_float(__float_as_int(a) ^ (int)(parity_word << 31));
}
__device__ __forceinline__ double flip(double a, uint32_t parity_word) {
    return __hiloint2double(__double2hiint(a) ^ (int)(parity_word << 31), __double2loint(a));
}

struct Geom {
    int nblk;
    int tile;
    int64_t cta_off[kMaxBlocks + 1];
    int64_t ntile[kMaxBlocks];
};

struct PlanDev {
    int32_t nbatch;
    const int32_t *b_i0, *it_g, *it_s0, *s_t0;
    const uint32_t *g_xlo, *g_xhi, *s_zlo, *s_xhi, *t_zhi;
    const double2 *t_c64;
    const float2 *t_c32;
};

struct Item {
    int64_t base;   // index of column 0 of the source row
    uint32_t xlo;   // group x mask, low half
    int klo;        // popcount the source column must have (-1: row invalid)
    int s0, s1;     // segment range in shared memory
};

template <typename R> __device__ __forceinline__ typename Cx<R>::T coef(const PlanDev &p, int t);
template <> __device__ __forceinline__ float2 coef<float>(const PlanDev &p, int t) { return p.t_c32[t]; }
template <> __device__ __forceinline__ double2 coef<double>(const PlanDev &p, int t) { return p.t_c64[t]; }

// Decode this CTA's (block, row, column tile).
struct RowCtx {
    int blk;
    uint32_t thi;
    int64_t own_base;
    int64_t dlo;
    int64_t c0;
};

template <bool FULL>
__device__ __forceinline__ RowCtx decode_row(const SectorView &v, const Geom &geo) {
    RowCtx rc;
    const int64_t cta = blockIdx.x;
    int b = 0;
    while (b + 1 < geo.nblk && geo.cta_off[b + 1] <= cta) ++b;
    const int64_t local = cta - geo.cta_off[b];
    const int64_t rowi = local / geo.ntile[b];
    const int64_t tile = local - rowi * geo.ntile[b];
    rc.blk = b;
    rc.dlo = v.dlo[b];
    rc.c0 = tile * geo.tile;
    if (FULL) {
        rc.thi = (uint32_t)rowi;
        rc.own_base = rowi << v.n_lo;
    } else {
        rc.thi = v.list_hi[v.list_hi_off[v.khi[b]] + rowi];
        rc.own_base = v.off[b] + rowi * v.dlo[b];
    }
    return rc;
}

template <typename R, bool FULL, bool REALH, int TPT>
__global__ void __launch_bounds__(kThreads)
k_apply(SectorView v, Geom geo, PlanDev p, const typename Cx<R>::T *__restrict__ psi,
        typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    using C2 = typename Cx<R>::T;
    __shared__ Item sm_item[PlanLimits::kGroupsPerBatch];
    __shared__ uint32_t sm_z[PlanLimits::kSegsPerBatch];
    __shared__ C2 sm_a[PlanLimits::kSegsPerBatch];

    const RowCtx rc = decode_row<FULL>(v, geo);
    const int tid = threadIdx.x;

    uint32_t tlo[TPT];
    bool act[TPT];
    R accr[TPT], acci[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        const int64_t c = rc.c0 + tid + j * kThreads;
        act[j] = c < rc.dlo;
        tlo[j] = 0;
        if (act[j]) tlo[j] = FULL ? (uint32_t)c : __ldg(v.list_lo + v.list_lo_off[v.klo[rc.blk]] + c);
        accr[j] = R(0);
        acci[j] = R(0);
    }

    for (int bt = 0; bt < p.nbatch; ++bt) {
        const int i0 = p.b_i0[bt], i1 = p.b_i0[bt + 1];
        const int s0 = p.it_s0[i0], s1 = p.it_s0[i1];
        // phase 1a: fold the row's high-half phases into one coefficient per segment
        for (int s = s0 + tid; s < s1; s += kThreads) {
            const uint32_t shi = rc.thi ^ __ldg(p.s_xhi + s);
            const bool ok = FULL || v.blk_of_khi[__popc(shi)] >= 0;
            R ar = R(0), ai = R(0);
            if (ok) {
                const int t1 = __ldg(p.s_t0 + s + 1);
                for (int t = __ldg(p.s_t0 + s); t < t1; ++t) {
                    const C2 c = coef<R>(p, t);
                    const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
                    ar += flip(c.x, par);
                    if (!REALH) ai += flip(c.y, par);
                }
            }
            C2 a;
            a.x = ar;
            a.y = ai;
            sm_a[s - s0] = a;
            sm_z[s - s0] = __ldg(p.s_zlo + s);
        }
        // phase 1b: per item, the source row of this CTA's row
        for (int it = i0 + tid; it < i1; it += kThreads) {
            const int g = __ldg(p.it_g + it);
            const uint32_t shi = rc.thi ^ __ldg(p.g_xhi + g);
            Item e;
            e.xlo = __ldg(p.g_xlo + g);
            e.s0 = __ldg(p.it_s0 + it) - s0;
            e.s1 = __ldg(p.it_s0 + it + 1) - s0;
            if (FULL) {
                e.klo = 0;
                e.base = (int64_t)shi << v.n_lo;
            } else {
                const int bb = v.blk_of_khi[__popc(shi)];
                if (bb < 0) {
                    e.klo = -1;
                    e.base = 0;
                } else {
                    e.klo = v.klo[bb];
                    e.base = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb];
                }
            }
            sm_item[it - i0] = e;
        }
        __syncthreads();
        // phase 2: gather
        const int nit = i1 - i0;
        for (int it = 0; it < nit; ++it) {
            const Item e = sm_item[it];
            if (e.klo < 0) continue;
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                if (!act[j]) continue;
                const uint32_t slo = tlo[j] ^ e.xlo;
                if (!FULL && __popc(slo) != e.klo) continue;
                const uint32_t r = FULL ? slo : __ldg(v.rank_lo + slo);
                const C2 amp = psi[e.base + r];
                R fr = R(0), fi = R(0);
                for (int s = e.s0; s < e.s1; ++s) {
                    const uint32_t par = __popc(sm_z[s] & slo);
                    const C2 a = sm_a[s];
                    fr += flip(a.x, par);
                    if (!REALH) fi += flip(a.y, par);
                }
                if (REALH) {
                    accr[j] += fr * amp.x;
                    acci[j] += fr * amp.y;
                } else {
                    accr[j] += fr * amp.x - fi * amp.y;
                    acci[j] += fr * amp.y + fi * amp.x;
                }
            }
        }
        __syncthreads();
    }

    // epilogue: store and / or FP64 reductions
    double er = 0.0, ei = 0.0, h2 = 0.0, p2 = 0.0;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t idx = rc.own_base + rc.c0 + tid + j * kThreads;
        if (flags & 1) {
            C2 o;
            o.x = accr[j];
            o.y = acci[j];
            out[idx] = o;
        }
        if (flags & 2) {
            const C2 ps = psi[idx];
            const double pr = (double)ps.x, pi = (double)ps.y;
            const double hr = (double)accr[j], hi = (double)acci[j];
            er += pr * hr + pi * hi;
            ei += pr * hi - pi * hr;
            h2 += hr * hr + hi * hi;
            p2 += pr * pr + pi * pi;
        }
    }
    if (flags & 2) {
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
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += red[tid][w];
            partials[(int64_t)blockIdx.x * 4 + tid] = s;
        }
    }
}

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

template <typename R, bool FULL>
__global__ void __launch_bounds__(kThreads)
k_rotate(SectorView v, Geom geo, int64_t m, uint64_t x, const uint64_t *__restrict__ z,
         const double2 *__restrict__ c, R theta, typename Cx<R>::T *psi, int *status) {
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
    if (act) tlo = FULL ? (uint32_t)col : __ldg(v.list_lo + v.list_lo_off[v.klo[rc.blk]] + col);
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
        const int bb = v.blk_of_khi[__popc(shi)];
        if (bb < 0 || __popc(slo) != v.klo[bb]) {
            if (fr != R(0) || fi != R(0)) atomicCAS(status, 0, (int)PAULI_ESECTOR);
            return;
        }
        sidx = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb] + (int64_t)__ldg(v.rank_lo + slo);
    }
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

Geom make_geom(const SectorView &v, int tile) {
    Geom g;
    g.nblk = v.nblk;
    g.tile = tile;
    g.cta_off[0] = 0;
    for (int b = 0; b < v.nblk; ++b) {
        const int64_t nt = (v.dlo[b] + tile - 1) / tile;
        g.ntile[b] = nt > 0 ? nt : 1;
        const int64_t ctas = (v.dlo[b] > 0) ? v.dhi[b] * nt : 0;
        g.cta_off[b + 1] = g.cta_off[b] + ctas;
    }
    return g;
}

int pick_tpt(const SectorView &v) {
    int64_t mx = 0;
    for (int b = 0; b < v.nblk; ++b) mx = std::max(mx, v.dlo[b]);
    if (mx >= 4 * kThreads) return 4;
    if (mx >= 2 * kThreads) return 2;
    return 1;
}

PlanDev plan_dev(const Plan &p) {
    PlanDev d;
    d.nbatch = (int32_t)p.nbatch;
    d.b_i0 = p.b_i0;
    d.it_g = p.it_g;
    d.it_s0 = p.it_s0;
    d.s_t0 = p.s_t0;
    d.g_xlo = p.g_xlo;
    d.g_xhi = p.g_xhi;
    d.s_zlo = p.s_zlo;
    d.s_xhi = p.s_xhi;
    d.t_zhi = p.t_zhi;
    d.t_c64 = p.t_c64;
    d.t_c32 = p.t_c32;
    return d;
}

template <typename R, bool FULL, bool REALH>
void launch_apply_t(int tpt, const SectorView &v, const Geom &geo, const PlanDev &pd, const void *in,
                    void *out, double *partials, int flags, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const int64_t nct = geo.cta_off[geo.nblk];
    if (nct == 0) return;
    PS_CHECK(nct < (1ll << 31), PAULI_EUNSUPPORTED, "apply: too many thread blocks");
    const C2 *pin = static_cast<const C2 *>(in);
    C2 *pout = static_cast<C2 *>(out);
    switch (tpt) {
        case 4: k_apply<R, FULL, REALH, 4><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
        case 2: k_apply<R, FULL, REALH, 2><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
        default: k_apply<R, FULL, REALH, 1><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
    }
    PS_LAUNCH_CHECK();
}

}  // namespace

int64_t apply_num_ctas(const Plan &p, const SectorView &v, int dtype) {
    (void)p;
    (void)dtype;
    const int tpt = pick_tpt(v);
    return make_geom(v, tpt * kThreads).cta_off[v.nblk];
}

void launch_apply(pauli_sum *H, const Plan &p, const SectorView &v, const void *psi_in, void *psi_out,
                  int dtype, double *partials, cudaStream_t st) {
    (void)H;
    const int tpt = pick_tpt(v);
    const Geom geo = make_geom(v, tpt * kThreads);
    const PlanDev pd = plan_dev(p);
    int flags = (psi_out ? 1 : 0) | (partials ? 2 : 0);
    const bool full = v.kind == PAULI_SECTOR_FULL;
    const bool real = p.real;
    if (dtype == PAULI_C64) {
        if (full) {
            if (real) launch_apply_t<float, true, true>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
            else launch_apply_t<float, true, false>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
        } else {
            if (real) launch_apply_t<float, false, true>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
            else launch_apply_t<float, false, false>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
        }
    } else {
        if (full) {
            if (real) launch_apply_t<double, true, true>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
            else launch_apply_t<double, true, false>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
        } else {
            if (real) launch_apply_t<double, false, true>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
            else launch_apply_t<double, false, false>(tpt, v, geo, pd, psi_in, psi_out, partials, flags, st);
        }
    }
}

void launch_reduce(const double *partials, int64_t nparts, double *result, cudaStream_t st) {
    k_reduce<<<1, 1024, 0, st>>>(partials, nparts, result);
    PS_LAUNCH_CHECK();
}

void launch_rotate(pauli_sum *G, const SectorView &v, double theta, void *psi, int dtype,
                   cudaStream_t st) {
    uint64_t x = 0;
    if (G->G == 1) PS_CUDA(cudaMemcpy(&x, G->gx, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const Geom geo = make_geom(v, kThreads);
    const int64_t nct = geo.cta_off[v.nblk];
    if (nct == 0) return;
    PS_CHECK(nct < (1ll << 31), PAULI_EUNSUPPORTED, "rotate: too many thread blocks");
    const bool full = v.kind == PAULI_SECTOR_FULL;
    if (dtype == PAULI_C64) {
        if (full) k_rotate<float, true><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, (float)theta, static_cast<float2 *>(psi), G->status);
        else k_rotate<float, false><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, (float)theta, static_cast<float2 *>(psi), G->status);
    } else {
        if (full) k_rotate<double, true><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, theta, static_cast<double2 *>(psi), G->status);
        else k_rotate<double, false><<<(unsigned)nct, kThreads, 0, st>>>(v, geo, G->m, x, G->z, G->c, theta, static_cast<double2 *>(psi), G->status);
    }
    PS_LAUNCH_CHECK();
}

}  // namespace ps
