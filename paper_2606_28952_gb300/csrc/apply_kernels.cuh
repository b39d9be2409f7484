// apply_kernels.cuh -- operator-state kernels of the gather family (Sec. 2.4):
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
#pragma once
#include <algorithm>
#include <cstdlib>

#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kThreads = 256;

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// (-1)^parity_word * a: the parity's low bit moved to the sign bit.  Adding it
// to the bit pattern equals the XOR (only bit 31 can change; the carry falls
// off) and issues as one integer add instead of a shift and a logic op
// (24-qubit molecule, complex64: 3.56 -> 3.29 ms per apply).
__device__ __forceinline__ float flip(float a, uint32_t parity_word) {
    return __int_as_float((int)((uint32_t)__float_as_int(a) + (parity_word << 31)));
}
__device__ __forceinline__ double flip(double a, uint32_t parity_word) {
    return __hiloint2double((int)((uint32_t)__double2hiint(a) + (parity_word << 31)), __double2loint(a));
}

// acc += f a for a real f: one packed FP32x2 FMA on the complex64 path (the same
// two fused multiply-adds as the scalar form)
__device__ __forceinline__ void fma_real(float2 &acc, float f, float2 a) { acc = __ffma2_rn(make_float2(f, f), a, acc); }
__device__ __forceinline__ void fma_real(double2 &acc, double f, double2 a) {
    acc.x = fma(f, a.x, acc.x);
    acc.y = fma(f, a.y, acc.y);
}

constexpr int kMaxSplit = 16;

struct Geom {
    int nblk;
    int tile;
    int64_t cta_off[kMaxBlocks + 1];
    int64_t ntile[kMaxBlocks];
    // each (row, column tile) is split into nsplit CTAs over consecutive piece
    // ranges [split_p0[k], split_p0[k+1]); their partial sums are added by k_combine
    int nsplit;
    int32_t split_p0[kMaxSplit + 1];
};

struct PlanDev {
    int32_t P, nseg_diag;
    const uint32_t *pc_xhi;
    const int32_t *pc_i0;
    const uint8_t *pc_lofree;
    const uint32_t *it_xlo;
    const uint32_t *it_xhi;
    const int32_t *it_s0;
    int32_t I;
    const uint32_t *s_zlo;
    const uint32_t *s_xhi;
    const int32_t *s_t0;
    int32_t S;
    const uint32_t *t_zhi;
    const double2 *t_c64;
    const float2 *t_c32;
    const double2 *diag_tab64;  // null: no diagonal table for this split
    const float2 *diag_tab32;
    const int32_t *diag_rest;
    int32_t n_diag_rest;
};

template <typename R> __device__ __forceinline__ typename Cx<R>::T coef(const PlanDev &p, int t);
template <> __device__ __forceinline__ float2 coef<float>(const PlanDev &p, int t) { return __ldg(p.t_c32 + t); }
template <> __device__ __forceinline__ double2 coef<double>(const PlanDev &p, int t) { return __ldg(p.t_c64 + t); }

// Decode this CTA's (block, row, column tile).
struct RowCtx {
    int blk;
    uint32_t thi;
    int64_t own_base;
    int64_t dlo;
    int64_t c0;
    int split;
};

template <bool FULL>
__device__ __forceinline__ RowCtx decode_row(const SectorView &v, const Geom &geo, int64_t work = -1) {
    RowCtx rc;
    if (work < 0) work = blockIdx.x;
    const int64_t cta = work / geo.nsplit;
    rc.split = (int)(work - cta * geo.nsplit);
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
        rc.thi = v.list_hi[v.lst_hi_off[b] + rowi];
        rc.own_base = v.off[b] + rowi * v.dlo[b];
    }
    return rc;
}

// cp.async (global -> shared, no register staging)
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Error-free sum (Knuth TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Per-thread sum of conj(x) y: FP64 on the FP64 path; on the FP32 path exact
// FP32 product splits summed with TwoSum, converted to FP64 once (as ExpAcc).
template <typename R> struct DotAcc;
template <> struct DotAcc<double> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(double2 x, double2 y) {
        re += x.x * y.x + x.y * y.y;
        im += x.x * y.y - x.y * y.x;
    }
    __device__ __forceinline__ double get_re() const { return re; }
    __device__ __forceinline__ double get_im() const { return im; }
};
template <> struct DotAcc<float> {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    __device__ __forceinline__ static void prod(float &s, float &c, float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float2 x, float2 y) {
        prod(sr, cr, x.x, y.x);
        prod(sr, cr, x.y, y.y);
        prod(si, ci, x.x, y.y);
        prod(si, ci, -x.y, y.x);
    }
    __device__ __forceinline__ double get_re() const { return (double)sr + (double)cr; }
    __device__ __forceinline__ double get_im() const { return (double)si + (double)ci; }
};

// Expectation partials of one thread's targets: {Re <psi|H psi>, Im, ||H psi||^2,
// <psi|psi>}.  FP64 path: FP64 products and sums.  FP32 path: every product is
// split exactly into FP32 hi + lo parts (FMA) and summed with TwoSum, so the
// few terms of a thread lose nothing; each pair becomes one FP64 number when
// the thread's partials enter the FP64 block reduction.  (FP64 arithmetic runs
// at a small fraction of the FP32 rate on this GPU.)
template <typename R> struct ExpAcc;
template <> struct ExpAcc<double> {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    __device__ __forceinline__ void add(double2 ps, double hr, double hi) {
        s[0] += ps.x * hr + ps.y * hi;
        s[1] += ps.x * hi - ps.y * hr;
        s[2] += hr * hr + hi * hi;
        s[3] += ps.x * ps.x + ps.y * ps.y;
    }
    __device__ __forceinline__ double get(int k) const { return s[k]; }
};
template <> struct ExpAcc<float> {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    __device__ __forceinline__ void prod(int k, float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float t, err;
        two_sum(s[k], p, t, err);
        s[k] = t;
        c[k] = __fadd_rn(c[k], __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float2 ps, float hr, float hi) {
        prod(0, ps.x, hr);
        prod(0, ps.y, hi);
        prod(1, ps.x, hi);
        prod(1, -ps.y, hr);
        prod(2, hr, hr);
        prod(2, hi, hi);
        prod(3, ps.x, ps.x);
        prod(3, ps.y, ps.y);
    }
    __device__ __forceinline__ double get(int k) const { return (double)s[k] + (double)c[k]; }
};

// KFULL: full space; KBLK1 / KBLKN: one / several product blocks, source rows
// staged by bit pattern (2^n_lo slots, zeros outside the block); KBLKR: one
// product block, source rows staged densely by rank and found through a rank
// table in shared memory (for splits too wide for 2^n_lo slots); KBLKC: KBLKN
// for point-group sectors, whose blocks are (popcount, irrep) classes.  Only
// KBLKC and KBLKR evaluate the class of a half-string (KBLKR once per row and
// rank table); the popcount kinds keep one POPC in their inner loops.
enum : int { KFULL = 0, KBLK1 = 1, KBLKN = 2, KBLKR = 3, KBLKC = 4 };

__host__ __device__ constexpr bool kind_multi(int k) { return k == KBLKN || k == KBLKC; }

template <int KIND>
__device__ __forceinline__ int kcls_lo(const SectorView &v, uint32_t s) {
    if constexpr (KIND == KBLKC || KIND == KBLKR) return cls_lo(v, s);
    else return __popc(s);
}
template <int KIND>
__device__ __forceinline__ int kcls_hi(const SectorView &v, uint32_t s) {
    if constexpr (KIND == KBLKC || KIND == KBLKR) return cls_hi(v, s);
    else return __popc(s);
}

// Rank table of KBLKR: n_lo <= 14: u16 lut[2^n_lo] (D_lo, the zero slot, for
// strings outside the block); 15..16: u32 tabA[256] (colex rank of the low
// byte) and tabB[256][9] (what the high byte adds, by the low byte's popcount).
__host__ __device__ inline size_t rank_table_bytes(int n_lo) {
    return n_lo <= 14 ? ((size_t)2 << n_lo) : (size_t)(256 + 256 * 9) * 4;
}
__host__ __device__ inline int ranked_rowcap(int64_t dlo) { return (int)((dlo + 2) & ~1ll); }

constexpr int kSegCap = PlanLimits::kSegsPerPiece;
constexpr int kItemCap = PlanLimits::kItemsPerPiece;

template <typename R>
struct Smem {
    using C2 = typename Cx<R>::T;
    // byte offsets inside one buffer
    // the low parts of the x = 0 group's coefficients exist on the FP32 path only
    static constexpr size_t kLoBytes = sizeof(R) == 4 ? sizeof(float2) : 0;
    static __host__ __device__ size_t buf_bytes(int rw) {
        return (size_t)rw * sizeof(C2) + (size_t)kSegCap * (sizeof(C2) + kLoBytes + 4) +
               (size_t)kItemCap * sizeof(int4);
    }
};

// One pipeline buffer: a staged source row (indexed by the low-half bit
// pattern, zero where the pattern is outside the source block), the piece's
// folded segment coefficients and its items.
template <typename R>
struct Buf {
    using C2 = typename Cx<R>::T;
    C2 *row;
    C2 *a;
    float2 *alo;   // low parts of the x = 0 group's coefficients (FP32 path only; no storage for FP64)
    int4 *item;    // {x_lo, seg begin, seg end, diagonal}
    uint32_t *z;
    __device__ Buf(char *base, int rw) {
        row = reinterpret_cast<C2 *>(base);
        a = reinterpret_cast<C2 *>(base + (size_t)rw * sizeof(C2));
        alo = reinterpret_cast<float2 *>(reinterpret_cast<char *>(a) + (size_t)kSegCap * sizeof(C2));
        item = reinterpret_cast<int4 *>(reinterpret_cast<char *>(alo) + (size_t)kSegCap * Smem<R>::kLoBytes);
        z = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(item) + (size_t)kItemCap * sizeof(int4));
    }
};

template <typename R, int KIND, bool REALH>
__device__ __forceinline__ void stage_piece(const SectorView &v, const PlanDev &p, int q, uint32_t thi,
                                            const typename Cx<R>::T *__restrict__ psi, Buf<R> &B,
                                            int *klo_req) {
    using C2 = typename Cx<R>::T;
    const int tid = threadIdx.x, nth = blockDim.x;
    const uint32_t shi = thi ^ __ldg(p.pc_xhi + q);
    int64_t base;
    int64_t len;
    int klo = 0;
    int64_t loff = 0;
    if (KIND == KFULL) {
        base = (int64_t)shi << v.n_lo;
        len = 1ll << v.n_lo;
    } else {
        const int bb = v.blk_of_khi[kcls_hi<KIND>(v, shi)];
        klo = v.klo[bb];
        loff = v.lst_lo_off[bb];
        base = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb];
        len = v.dlo[bb];
    }
    // 1. source row -> shared memory, asynchronously
    if (KIND == KFULL) {
        if (sizeof(C2) == 16) {
            for (int64_t r = tid; r < len; r += nth) cp_async16(B.row + r, psi + base + r);
        } else {
            for (int64_t r = 2 * tid; r < len; r += 2 * nth) cp_async16(B.row + r, psi + base + r);
        }
    } else if (KIND == KBLKR) {
        // dense copy of the source row, indexed later through the rank table; on the
        // complex64 path two amplitudes per 16-byte copy when the row starts on an
        // even index (every row of an even-width block)
        if (sizeof(C2) == 16) {
            for (int64_t r = tid; r < len; r += nth) cp_async16(B.row + r, psi + base + r);
        } else if ((base & 1) == 0) {
            for (int64_t r = 2 * tid; r + 1 < len; r += 2 * nth) cp_async16(B.row + r, psi + base + r);
            if ((len & 1) && tid == 0) cp_async8(B.row + len - 1, psi + base + len - 1);
        } else {
            for (int64_t r = tid; r < len; r += nth) cp_async8(B.row + r, psi + base + r);
        }
    } else {
        const uint32_t *lst = v.list_lo + loff;
        for (int64_t r = tid; r < len; r += nth) {
            const uint32_t pos = __ldg(lst + r);
            if (sizeof(C2) == 16) cp_async16(B.row + pos, psi + base + r);
            else cp_async8(B.row + pos, psi + base + r);
        }
    }
    cp_async_commit();
    // 2. items of the piece
    const int i0 = __ldg(p.pc_i0 + q), i1 = __ldg(p.pc_i0 + q + 1);
    const int sbase = __ldg(p.it_s0 + i0);
    for (int it = i0 + tid; it < i1; it += nth) {
        const int s0 = __ldg(p.it_s0 + it), s1 = __ldg(p.it_s0 + it + 1);
        B.item[it - i0] = make_int4((int)__ldg(p.it_xlo + it), s0 - sbase, s1 - sbase, s0 < p.nseg_diag ? 1 : 0);
    }
    // 3. fold the high-half phases of this row into one coefficient per segment
    const int send = __ldg(p.it_s0 + i1);
    for (int s = sbase + tid; s < send; s += nth) {
        const int t0 = __ldg(p.s_t0 + s), t1 = __ldg(p.s_t0 + s + 1);
        C2 a;
        float2 lo = make_float2(0.f, 0.f);
        if (sizeof(R) == 4 && s < p.nseg_diag) {
            // x = 0 group on the FP32 path: sum in FP64, keep the rounding residue
            double ar = 0.0, ai = 0.0;
            for (int t = t0; t < t1; ++t) {
                const double2 c = __ldg(p.t_c64 + t);
                const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
                ar += flip(c.x, par);
                ai += flip(c.y, par);
            }
            a.x = (R)ar;
            a.y = (R)ai;
            lo = make_float2((float)(ar - (double)(float)ar), (float)(ai - (double)(float)ai));
        } else {
            R ar = R(0), ai = R(0);
            for (int t = t0; t < t1; ++t) {
                const C2 c = coef<R>(p, t);
                const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
                ar += flip(c.x, par);
                if (!REALH) ai += flip(c.y, par);
            }
            a.x = ar;
            a.y = ai;
        }
        B.a[s - sbase] = a;
        if (sizeof(R) == 4) B.alo[s - sbase] = lo;
        B.z[s - sbase] = __ldg(p.s_zlo + s);
    }
    if (kind_multi(KIND) && tid == 0) *klo_req = klo;
}

template <typename R, int KIND>
__device__ __forceinline__ int next_piece(const SectorView &v, const PlanDev &p, int q, uint32_t thi, int pend) {
    for (++q; q < pend; ++q) {
        if (KIND == KFULL) break;
        const uint32_t shi = thi ^ __ldg(p.pc_xhi + q);
        if (v.blk_of_khi[kcls_hi<KIND>(v, shi)] >= 0) break;
    }
    return q;
}

// Rank lookup of KBLKR (see rank_table_bytes).
struct RankTab {
    const uint16_t *lut;
    const uint32_t *tabA, *tabB;
    int n_lo, klo;
    uint32_t dlo;
};

__device__ __forceinline__ uint32_t ranked_index(const RankTab &rt, uint32_t s) {
    if (rt.n_lo <= 14) return rt.lut[s];
    const uint32_t lo8 = s & 255u;
    const uint32_t r = rt.tabA[lo8] + rt.tabB[(s >> 8) * 9 + __popc(lo8)];
    return __popc(s) == rt.klo ? r : rt.dlo;
}

// NJ <= TPT: the columns j < NJ are evaluated (a warp whose last column lies
// beyond the row runs with NJ = TPT - 1 and skips that column's work)
template <typename R, int KIND, bool REALH, int TPT, int NJ = TPT>
__device__ __forceinline__ void gather_piece(const SectorView &v, const PlanDev &p, int q, const Buf<R> &B, int klo_req,
                                             const uint32_t (&tlo)[TPT], R (&accr)[TPT], R (&acci)[TPT],
                                             const RankTab &rt) {
    using C2 = typename Cx<R>::T;
    const int nit = __ldg(p.pc_i0 + q + 1) - __ldg(p.pc_i0 + q);
    for (int it = 0; it < nit; ++it) {
        const int4 e = B.item[it];
        uint32_t s[TPT];
#pragma unroll
        for (int j = 0; j < NJ; ++j) s[j] = tlo[j] ^ (uint32_t)e.x;
        R fr[TPT], fi[TPT];
        // the staged-row loads go out before the segment sums so that their
        // shared-memory latency overlaps them (24-qubit molecule 2.56 -> 2.52 ms,
        // 64 batched molecules 0.97 -> 0.90 s)
        C2 amp0[TPT];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            fr[j] = R(0);
            fi[j] = R(0);
            amp0[j] = B.row[(KIND == KBLKR) ? ranked_index(rt, s[j]) : s[j]];
        }
        if (sizeof(R) == 4 && e.w) {
            // x = 0 group: compensated FP32 summation of hi / lo coefficient pairs
            R er[TPT], ei[TPT];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                er[j] = R(0);
                ei[j] = R(0);
            }
            for (int sg = e.y; sg < e.z; ++sg) {
                const uint32_t z = B.z[sg];
                const C2 a = B.a[sg];
                const float2 l = B.alo[sg];
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const uint32_t par = __popc(z & s[j]);
                    float t, err;
                    two_sum(fr[j], flip((float)a.x, par), t, err);
                    fr[j] = t;
                    er[j] += err + flip(l.x, par);
                    if (!REALH) {
                        two_sum(fi[j], flip((float)a.y, par), t, err);
                        fi[j] = t;
                        ei[j] += err + flip(l.y, par);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                fr[j] += er[j];
                fi[j] += ei[j];
            }
        } else {
#pragma unroll 2
            for (int sg = e.y; sg < e.z; ++sg) {
                const uint32_t z = B.z[sg];
                const C2 a = B.a[sg];
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const uint32_t par = __popc(z & s[j]);
                    fr[j] += flip(a.x, par);
                    if (!REALH) fi[j] += flip(a.y, par);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            C2 amp = amp0[j];
            if (kind_multi(KIND) && kcls_lo<KIND>(v, s[j]) != klo_req) {
                amp.x = R(0);
                amp.y = R(0);
            }
            if (REALH) {
                accr[j] += fr[j] * amp.x;
                acci[j] += fr[j] * amp.y;
            } else {
                accr[j] += fr[j] * amp.x - fi[j] * amp.y;
                acci[j] += fr[j] * amp.y + fi[j] * amp.x;
            }
        }
    }
}

// A piece whose items all have x_lo = 0 (none of the x = 0 group) reads each
// target's source in the same column of the source row.  Every thread folds
// the piece's high-half phases into the segment coefficients itself (the same
// loads across the CTA, served by L1) and reads psi from global memory: no
// staging and no barrier.  Sources of a full space or of a single block only.
template <typename R, int KIND, bool REALH, int TPT, int NJ = TPT>
__device__ __forceinline__ void lofree_piece(const SectorView &v, const PlanDev &p, int q, uint32_t thi,
                                             const typename Cx<R>::T *__restrict__ psi, int64_t c0,
                                             const bool (&act)[TPT], const uint32_t (&tlo)[TPT], R (&accr)[TPT],
                                             R (&acci)[TPT]) {
    using C2 = typename Cx<R>::T;
    const uint32_t shi = thi ^ __ldg(p.pc_xhi + q);
    int64_t base;
    if (KIND == KFULL) {
        base = (int64_t)shi << v.n_lo;
    } else {
        const int bb = v.blk_of_khi[kcls_hi<KIND>(v, shi)];
        base = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb];
    }
    C2 amp[TPT];
    R fr[TPT], fi[TPT];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        amp[j].x = R(0);
        amp[j].y = R(0);
        if (act[j]) amp[j] = psi[base + c0 + threadIdx.x + j * kThreads];
        fr[j] = R(0);
        fi[j] = R(0);
    }
    const int s0 = __ldg(p.it_s0 + __ldg(p.pc_i0 + q)), s1 = __ldg(p.it_s0 + __ldg(p.pc_i0 + q + 1));
    for (int s = s0; s < s1; ++s) {
        const int t0 = __ldg(p.s_t0 + s), t1 = __ldg(p.s_t0 + s + 1);
        R ar = R(0), ai = R(0);
        for (int t = t0; t < t1; ++t) {
            const C2 c = coef<R>(p, t);
            const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
            ar += flip(c.x, par);
            if (!REALH) ai += flip(c.y, par);
        }
        const uint32_t z = __ldg(p.s_zlo + s);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            const uint32_t par = __popc(z & tlo[j]);
            fr[j] += flip(ar, par);
            if (!REALH) fi[j] += flip(ai, par);
        }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        if (REALH) {
            accr[j] += fr[j] * amp[j].x;
            acci[j] += fr[j] * amp[j].y;
        } else {
            accr[j] += fr[j] * amp[j].x - fi[j] * amp[j].y;
            acci[j] += fr[j] * amp[j].y + fi[j] * amp[j].x;
        }
    }
}

// One (row, column tile, piece range) work unit of the staged gather; the body
// of k_apply and of the persistent batched launch.  part4: this unit's 4 FP64
// expectation partials (flags & 2).
template <typename R, int KIND, bool REALH, int TPT, int NBUF>
__device__ __forceinline__ void apply_unit(const SectorView &v, const Geom &geo, const PlanDev &p, int64_t work,
                                           const typename Cx<R>::T *__restrict__ psi,
                                           typename Cx<R>::T *__restrict__ out, double *__restrict__ part4,
                                           int flags, char *smem) {
    using C2 = typename Cx<R>::T;
    __shared__ int klo_req[2];
    const int rw = (KIND == KBLKR) ? ranked_rowcap(v.dlo[0]) : (1 << v.n_lo);
    const size_t bb = Smem<R>::buf_bytes(rw);
    Buf<R> B0(smem, rw), B1(smem + (NBUF > 1 ? bb : 0), rw);
    const RowCtx rc = decode_row<KIND == KFULL>(v, geo, work);
    const int tid = threadIdx.x;

    RankTab rt;
    rt.lut = nullptr;
    rt.tabA = rt.tabB = nullptr;
    rt.n_lo = v.n_lo;
    rt.klo = v.klo[0];
    rt.dlo = (uint32_t)v.dlo[0];
    if (KIND == KBLKR) {
        char *tab = smem + (size_t)NBUF * bb;
        rt.lut = reinterpret_cast<const uint16_t *>(tab);
        rt.tabA = reinterpret_cast<const uint32_t *>(tab);
        rt.tabB = rt.tabA + 256;
        const int klo = v.klo[0];
        const int64_t dlo = v.dlo[0];
        if (v.n_lo <= 14) {
            uint16_t *lut = reinterpret_cast<uint16_t *>(tab);
            for (int s = tid; s < (1 << v.n_lo); s += kThreads)
                lut[s] = (uint16_t)(cls_lo(v, (uint32_t)s) == klo ? __ldg(v.rank_lo + s) : (uint32_t)dlo);
        } else {
            uint32_t *tabA = reinterpret_cast<uint32_t *>(tab);
            uint32_t *tabB = tabA + 256;
            for (int s = tid; s < 256; s += kThreads) tabA[s] = __ldg(v.rank_lo + s);
            for (int e = tid; e < 256 * 9; e += kThreads) {
                const uint32_t h = (uint32_t)(e / 9), k0 = (uint32_t)(e % 9);
                const uint32_t s = (h << 8) | ((1u << k0) - 1u);
                tabB[e] = (h < (1u << (v.n_lo - 8))) ? __ldg(v.rank_lo + s) : 0u;
            }
        }
        C2 zz;
        zz.x = R(0);
        zz.y = R(0);
        if (tid == 0) {
            B0.row[dlo] = zz;  // the zero slot
            if (NBUF > 1) B1.row[dlo] = zz;
        }
    } else if (KIND != KFULL) {
        // slots outside the source block stay zero
        for (int r = tid; r < rw; r += kThreads) {
            C2 zz;
            zz.x = R(0);
            zz.y = R(0);
            B0.row[r] = zz;
            if (NBUF > 1) B1.row[r] = zz;
        }
    }
    uint32_t tlo[TPT];
    bool act[TPT];
    R accr[TPT], acci[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        const int64_t c = rc.c0 + tid + j * kThreads;
        act[j] = c < rc.dlo;
        tlo[j] = 0;
        if (act[j]) tlo[j] = (KIND == KFULL) ? (uint32_t)c : __ldg(v.list_lo + v.lst_lo_off[rc.blk] + c);
        accr[j] = R(0);
        acci[j] = R(0);
    }
    __syncthreads();
    // four columns a thread: a warp whose fourth column is past the row's end for
    // every lane (e.g. D_lo = 924 against 1,024 slots) skips that column's work
    constexpr int NJS = TPT == 4 ? 3 : TPT;
    const bool short_warp = TPT == 4 && !__any_sync(0xffffffffu, act[TPT - 1]);

    const int pend = geo.split_p0[rc.split + 1];
    int q = next_piece<R, KIND>(v, p, geo.split_p0[rc.split] - 1, rc.thi, pend);
    if (NBUF > 1) {
        int c = 0;
        if (q < pend) stage_piece<R, KIND, REALH>(v, p, q, rc.thi, psi, B0, &klo_req[0]);
        while (q < pend) {
            const int qn = next_piece<R, KIND>(v, p, q, rc.thi, pend);
            if (qn < pend) {
                stage_piece<R, KIND, REALH>(v, p, qn, rc.thi, psi, c ? B0 : B1, &klo_req[c ^ 1]);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            if (short_warp) gather_piece<R, KIND, REALH, TPT, NJS>(v, p, q, c ? B1 : B0, klo_req[c], tlo, accr, acci, rt);
            else gather_piece<R, KIND, REALH, TPT>(v, p, q, c ? B1 : B0, klo_req[c], tlo, accr, acci, rt);
            __syncthreads();
            c ^= 1;
            q = qn;
        }
    } else {
        while (q < pend) {
            if (!kind_multi(KIND) && __ldg(p.pc_lofree + q)) {
                if (short_warp) lofree_piece<R, KIND, REALH, TPT, NJS>(v, p, q, rc.thi, psi, rc.c0, act, tlo, accr, acci);
                else lofree_piece<R, KIND, REALH, TPT>(v, p, q, rc.thi, psi, rc.c0, act, tlo, accr, acci);
            } else {
                stage_piece<R, KIND, REALH>(v, p, q, rc.thi, psi, B0, &klo_req[0]);
                cp_async_wait<0>();
                __syncthreads();
                if (short_warp) gather_piece<R, KIND, REALH, TPT, NJS>(v, p, q, B0, klo_req[0], tlo, accr, acci, rt);
                else gather_piece<R, KIND, REALH, TPT>(v, p, q, B0, klo_req[0], tlo, accr, acci, rt);
                __syncthreads();
            }
            q = next_piece<R, KIND>(v, p, q, rc.thi, pend);
        }
    }

    // epilogue: store and / or FP64 reductions
    ExpAcc<R> ea;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t idx = rc.own_base + rc.c0 + tid + j * kThreads;
        if (flags & 1) {
            C2 o;
            o.x = accr[j];
            o.y = acci[j];
            // split launches write partial sums to slice `split` of the scratch
            out[(flags & 4) ? (int64_t)rc.split * v.dim + idx : idx] = o;
        }
        if (flags & 2) ea.add(psi[idx], accr[j], acci[j]);
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
            part4[tid] = sum;
        }
    }
}

// Register budgets: four or more FP32 columns a thread take the budget of
// four resident CTAs (64 registers a thread) where the compiler's own choice
// spills (a complex operator, or two staged rows); the real operator with one
// staged row (64 registers by itself, and measurably faster without the
// bound) and every other instantiation keep the compiler's own allocation
// (a minimum of 0 CTAs per SM states no bound).
template <typename R, int KIND, bool REALH, int TPT, int NBUF>
__global__ void __launch_bounds__(kThreads, (sizeof(R) == 4 && TPT >= 4 && !(REALH && NBUF == 1)) ? 4 : 0)
k_apply(SectorView v, Geom geo, PlanDev p, const typename Cx<R>::T *__restrict__ psi,
        typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    extern __shared__ __align__(16) char smem[];
    apply_unit<R, KIND, REALH, TPT, NBUF>(v, geo, p, blockIdx.x, psi, out,
                                          partials ? partials + (int64_t)blockIdx.x * 4 : nullptr, flags, smem);
}

// The same body for rank-staged rows: their shared-memory rows leave one or two
// CTAs per SM, so the register budget is that of one resident CTA (without the
// bound the compiler keeps to ~40 registers and spills; measured on the 32-qubit
// sector: 7.27 s -> 5.01 s per apply together with 8 columns per thread).  The
// other gathers keep the compiler's choice, which measured faster there than a
// spill-free five- or four-CTA budget.
template <typename R, int KIND, bool REALH, int TPT, int NBUF>
__global__ void __launch_bounds__(kThreads, 1)
k_apply_wide(SectorView v, Geom geo, PlanDev p, const typename Cx<R>::T *__restrict__ psi,
             typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    extern __shared__ __align__(16) char smem[];
    apply_unit<R, KIND, REALH, TPT, NBUF>(v, geo, p, blockIdx.x, psi, out,
                                          partials ? partials + (int64_t)blockIdx.x * 4 : nullptr, flags, smem);
}

// ---------------------------------------------------------------------------
// Persistent batched launch: one grid of (#SM x resident) CTAs pulls work
// units -- (state, row, column tile) -- from an atomic queue; states are
// ordered largest first.  Every output element is still written by exactly
// one thread (the queue counter is the only atomic); each state's FP64
// expectation partials land in its own slice and are reduced in a fixed order.
// ---------------------------------------------------------------------------
struct BatchDesc {
    SectorView v;
    Geom geo;
    PlanDev p;
    int64_t work0;      // first work unit of this state in the queue order
    int64_t nwork;
    int64_t part0;      // first 4-double partial slot of this state
};

struct BatchPtrs {
    const void *in;
    void *out;          // may be null (expectation only)
};

template <typename R, int KIND, bool REALH, int TPT, int NBUF>
__global__ void __launch_bounds__(kThreads)
k_apply_batch(const BatchDesc *__restrict__ descs, const BatchPtrs *__restrict__ ptrs, int nstates,
              int64_t total, unsigned long long *counter, double *__restrict__ partials, int want_out) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) char smem[];
    __shared__ long long s_work;
    for (;;) {
        if (threadIdx.x == 0) s_work = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t work = s_work;
        __syncthreads();
        if (work >= total) break;
        int lo = 0, hi = nstates - 1;  // last state with work0 <= work
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].work0 <= work) lo = mid;
            else hi = mid - 1;
        }
        const BatchDesc &d = descs[lo];
        const BatchPtrs bp = ptrs[lo];
        const int64_t local = work - d.work0;
        const int flags = ((want_out && bp.out) ? 1 : 0) | 2;
        apply_unit<R, KIND, REALH, TPT, NBUF>(d.v, d.geo, d.p, local, static_cast<const C2 *>(bp.in),
                                               static_cast<C2 *>(bp.out), partials + (d.part0 + local) * 4, flags,
                                               smem);
    }
}

// results[b][0..3] = fixed-order sum of state b's partials
__global__ void __launch_bounds__(256) k_batch_reduce(const BatchDesc *__restrict__ descs, const double *partials,
                                                      double *results) {
    __shared__ double sm[4][256];
    const BatchDesc &d = descs[blockIdx.x];
    const int t = threadIdx.x;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = t; i < d.nwork; i += 256)
        for (int k = 0; k < 4; ++k) s[k] += partials[(d.part0 + i) * 4 + k];
    for (int k = 0; k < 4; ++k) sm[k][t] = s[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < 4; ++k) sm[k][t] += sm[k][t + o];
        __syncthreads();
    }
    if (t < 4) results[(int64_t)blockIdx.x * 4 + t] = sm[t][0];
}


// ---------------------------------------------------------------------------
// Direct variant for small operators (few groups per row, e.g. lattice models):
// the whole plan, folded for this CTA's row, lives in shared memory and every
// source amplitude is read straight from global memory (coalesced along a row
// of the full space), so a row costs one barrier instead of one per piece.
// ---------------------------------------------------------------------------
constexpr int kDirectItems = 256;
constexpr int kDirectSegs = 1024;

struct DItem {
    int64_t base;   // index of column 0 of the source row
    uint32_t xlo;
    int klo;        // popcount required of the source column, -1: row invalid
    int s0, s1;     // segment range (the first is skipped into f0 when its z_lo == 0)
    int diag;       // x = 0 group on the FP32 path: compensated sum
    int x0;         // x = 0 group (either path)
};

template <typename R, int KIND, bool REALH, int TPT>
__global__ void __launch_bounds__(kThreads, 4)
k_apply_direct(SectorView v, Geom geo, PlanDev p, const typename Cx<R>::T *__restrict__ psi,
               typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    using C2 = typename Cx<R>::T;
    __shared__ DItem sm_it[kDirectItems];
    __shared__ uint32_t sm_z[kDirectSegs];
    __shared__ C2 sm_a[kDirectSegs];
    __shared__ float2 sm_lo[kDirectSegs];
    const RowCtx rc = decode_row<KIND == KFULL>(v, geo);
    const int tid = threadIdx.x;
    // phase 1a: the source row of every item for this CTA's row
    for (int it = tid; it < p.I; it += kThreads) {
        const uint32_t shi = rc.thi ^ __ldg(p.it_xhi + it);
        const int s0 = __ldg(p.it_s0 + it), s1 = __ldg(p.it_s0 + it + 1);
        DItem e;
        e.xlo = __ldg(p.it_xlo + it);
        e.s0 = s0;
        e.s1 = s1;
        e.diag = (sizeof(R) == 4 && s0 < p.nseg_diag) ? 1 : 0;
        e.x0 = s0 < p.nseg_diag ? 1 : 0;
        if (KIND == KFULL) {
            e.klo = 0;
            e.base = (int64_t)shi << v.n_lo;
        } else {
            const int bb = v.blk_of_khi[kcls_hi<KIND>(v, shi)];
            e.klo = bb < 0 ? -1 : v.klo[bb];
            e.base = bb < 0 ? 0 : v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb];
        }
        sm_it[it] = e;
    }
    // phase 1b: one thread per segment folds the row's high-half phases (with
    // a diagonal table, the tabulated z_hi = 0 term of a diagonal segment is left out)
    const bool use_tab = p.diag_tab64 != nullptr;
    for (int s = tid; s < p.S; s += kThreads) {
        const uint32_t shi = rc.thi ^ __ldg(p.s_xhi + s);
        int t0 = __ldg(p.s_t0 + s);
        const int t1 = __ldg(p.s_t0 + s + 1);
        if (use_tab && s < p.nseg_diag && __ldg(p.t_zhi + t0) == 0u) ++t0;
        C2 a;
        float2 lo = make_float2(0.f, 0.f);
        if (sizeof(R) == 4 && s < p.nseg_diag) {
            double ar = 0.0, ai = 0.0;
            for (int t = t0; t < t1; ++t) {
                const double2 c = __ldg(p.t_c64 + t);
                const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
                ar += flip(c.x, par);
                ai += flip(c.y, par);
            }
            a.x = (R)ar;
            a.y = (R)ai;
            lo = make_float2((float)(ar - (double)(float)ar), (float)(ai - (double)(float)ai));
        } else {
            R ar = R(0), ai = R(0);
            for (int t = t0; t < t1; ++t) {
                const C2 c = coef<R>(p, t);
                const uint32_t par = __popc(__ldg(p.t_zhi + t) & shi);
                ar += flip(c.x, par);
                if (!REALH) ai += flip(c.y, par);
            }
            a.x = ar;
            a.y = ai;
        }
        sm_a[s] = a;
        sm_lo[s] = lo;
        sm_z[s] = __ldg(p.s_zlo + s);
    }
    uint32_t tlo[TPT];
    bool act[TPT];
    C2 acc[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        const int64_t c = rc.c0 + tid + j * kThreads;
        act[j] = c < rc.dlo;
        tlo[j] = 0;
        if (act[j]) tlo[j] = (KIND == KFULL) ? (uint32_t)c : __ldg(v.list_lo + v.lst_lo_off[rc.blk] + c);
        acc[j].x = R(0);
        acc[j].y = R(0);
    }
    __syncthreads();
    // phase 2: gather from global memory
    const bool full_tile = rc.c0 + (int64_t)TPT * kThreads <= rc.dlo;  // every column of the tile exists
    const int own_cls = KIND == KFULL ? 0 : v.klo[rc.blk];             // low-half class of this row's columns
    for (int it = 0; it < p.I; ++it) {
        const DItem e = sm_it[it];
        if (e.klo < 0) continue;
        uint32_t s[TPT];
        C2 amp[TPT];
        // x_lo = 0 on a block sector: the source column is the target's own.  Within the
        // same low-half class its rank is the column index (no class test, no rank
        // lookup); in another class no column of this row has a source in the block.
        // (real coefficients only: on the complex path the extra branch costs spills)
        const bool same_col = REALH && KIND != KFULL && e.xlo == 0u;
        if (same_col && e.klo != own_cls) continue;
        if (same_col) {
            const C2 *src = psi + (e.base + rc.c0 + tid);
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                s[j] = tlo[j];
                if (act[j]) {
                    amp[j] = src[j * kThreads];
                } else {
                    amp[j].x = R(0);
                    amp[j].y = R(0);
                }
            }
        } else if (KIND == KFULL) {
            // full space: the source row is contiguous; 32-bit offsets into it
            const C2 *src = psi + e.base;
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                s[j] = tlo[j] ^ e.xlo;
                amp[j] = src[s[j]];
            }
            if (!full_tile) {
#pragma unroll
                for (int j = 0; j < TPT; ++j)
                    if (!act[j]) {
                        amp[j].x = R(0);
                        amp[j].y = R(0);
                    }
            }
        } else {
            const C2 *src = psi + e.base;  // the source row; 32-bit ranks into it
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                s[j] = tlo[j] ^ e.xlo;
                const bool ok = act[j] && (kcls_lo<KIND>(v, s[j]) == e.klo);
                amp[j] = src[ok ? __ldg(v.rank_lo + s[j]) : 0u];
                if (!ok) {
                    amp[j].x = R(0);
                    amp[j].y = R(0);
                }
            }
        }
        R fr[TPT], fi[TPT];
        if (use_tab && e.x0) {
            // x = 0 group: table of the z_hi = 0 terms plus the remaining segments
            if (e.s0 != 0) continue;  // later items of a split diagonal group are covered here
            const uint32_t ntab = 1u << v.n_lo;
            if (sizeof(R) == 4) {
                R er[TPT], ei[TPT];
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const float2 h = __ldg(p.diag_tab32 + s[j]);
                    const float2 l = __ldg(p.diag_tab32 + ntab + s[j]);
                    fr[j] = (R)h.x;
                    fi[j] = (R)h.y;
                    er[j] = (R)l.x;
                    ei[j] = (R)l.y;
                }
                for (int r = 0; r < p.n_diag_rest; ++r) {
                    const int sgr = __ldg(p.diag_rest + r);
                    const uint32_t z = sm_z[sgr];
                    const C2 a = sm_a[sgr];
                    const float2 l = sm_lo[sgr];
#pragma unroll
                    for (int j = 0; j < TPT; ++j) {
                        const uint32_t par = __popc(z & s[j]);
                        float t, err;
                        two_sum(fr[j], flip((float)a.x, par), t, err);
                        fr[j] = t;
                        er[j] += err + flip(l.x, par);
                        if (!REALH) {
                            two_sum(fi[j], flip((float)a.y, par), t, err);
                            fi[j] = t;
                            ei[j] += err + flip(l.y, par);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    fr[j] += er[j];
                    fi[j] += ei[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const double2 h = __ldg(p.diag_tab64 + s[j]);
                    fr[j] = (R)h.x;
                    fi[j] = (R)h.y;
                }
                for (int r = 0; r < p.n_diag_rest; ++r) {
                    const int sgr = __ldg(p.diag_rest + r);
                    const uint32_t z = sm_z[sgr];
                    const C2 a = sm_a[sgr];
#pragma unroll
                    for (int j = 0; j < TPT; ++j) {
                        const uint32_t par = __popc(z & s[j]);
                        fr[j] += flip(a.x, par);
                        if (!REALH) fi[j] += flip(a.y, par);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                if (REALH) {
                    fma_real(acc[j], fr[j], amp[j]);
                } else {
                    acc[j].x += fr[j] * amp[j].x - fi[j] * amp[j].y;
                    acc[j].y += fr[j] * amp[j].y + fi[j] * amp[j].x;
                }
            }
            continue;
        }
        int sg = e.s0;
        const bool zfirst = sm_z[e.s0] == 0;
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            fr[j] = zfirst ? sm_a[e.s0].x : R(0);
            fi[j] = zfirst ? sm_a[e.s0].y : R(0);
        }
        if (zfirst) ++sg;
        if (sizeof(R) == 4 && e.diag) {
            R er[TPT], ei[TPT];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                er[j] = zfirst ? (R)sm_lo[e.s0].x : R(0);
                ei[j] = zfirst ? (R)sm_lo[e.s0].y : R(0);
            }
            for (; sg < e.s1; ++sg) {
                const uint32_t z = sm_z[sg];
                const C2 a = sm_a[sg];
                const float2 l = sm_lo[sg];
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const uint32_t par = __popc(z & s[j]);
                    float t, err;
                    two_sum(fr[j], flip((float)a.x, par), t, err);
                    fr[j] = t;
                    er[j] += err + flip(l.x, par);
                    if (!REALH) {
                        two_sum(fi[j], flip((float)a.y, par), t, err);
                        fi[j] = t;
                        ei[j] += err + flip(l.y, par);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                fr[j] += er[j];
                fi[j] += ei[j];
            }
        } else {
            for (; sg < e.s1; ++sg) {
                const uint32_t z = sm_z[sg];
                const C2 a = sm_a[sg];
#pragma unroll
                for (int j = 0; j < TPT; ++j) {
                    const uint32_t par = __popc(z & s[j]);
                    fr[j] += flip(a.x, par);
                    if (!REALH) fi[j] += flip(a.y, par);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < TPT; ++j) {
            if (REALH) {
                fma_real(acc[j], fr[j], amp[j]);
            } else {
                acc[j].x += fr[j] * amp[j].x - fi[j] * amp[j].y;
                acc[j].y += fr[j] * amp[j].y + fi[j] * amp[j].x;
            }
        }
    }
    // epilogue (same contract as k_apply)
    ExpAcc<R> ea;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t idx = rc.own_base + rc.c0 + tid + j * kThreads;
        if (flags & 1) out[idx] = acc[j];
        if (flags & 2) ea.add(psi[idx], acc[j].x, acc[j].y);
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
}

// out[i] = sum_k part[k][i] in a fixed order, then (optionally) the FP64
// expectation partial sums of pauli_expect for this block's elements.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_combine(int nsplit, int64_t dim, const typename Cx<R>::T *__restrict__ part, const typename Cx<R>::T *__restrict__ psi,
          typename Cx<R>::T *__restrict__ out, double *__restrict__ partials, int flags) {
    using C2 = typename Cx<R>::T;
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    ExpAcc<R> ea;
    if (i < dim) {
        C2 s = part[i];
        for (int k = 1; k < nsplit; ++k) {
            const C2 t = part[(int64_t)k * dim + i];
            s.x += t.x;
            s.y += t.y;
        }
        if (flags & 1) out[i] = s;
        if (flags & 2) ea.add(psi[i], s.x, s.y);
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
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][warp] = er;
            red[1][warp] = ei;
            red[2][warp] = h2;
            red[3][warp] = p2;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            double sum = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) sum += red[threadIdx.x][w];
            partials[(int64_t)blockIdx.x * 4 + threadIdx.x] = sum;
        }
    }
}

Geom make_geom(const SectorView &v, int tile, int nsplit = 1, const int32_t *split_p0 = nullptr,
               int32_t npieces = 0) {
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
    g.nsplit = nsplit;
    g.split_p0[0] = 0;
    g.split_p0[1] = npieces;
    if (split_p0)
        for (int k = 0; k <= nsplit; ++k) g.split_p0[k] = split_p0[k];
    return g;
}

PlanDev plan_dev(const Plan &p) {
    PlanDev d;
    d.P = (int32_t)p.P;
    d.nseg_diag = p.nseg_diag;
    d.pc_xhi = p.pc_xhi;
    d.pc_i0 = p.pc_i0;
    d.pc_lofree = p.pc_lofree;
    d.it_xlo = p.it_xlo;
    d.it_xhi = p.it_xhi;
    d.it_s0 = p.it_s0;
    d.I = (int32_t)p.I;
    d.s_zlo = p.s_zlo;
    d.s_xhi = p.s_xhi;
    d.s_t0 = p.s_t0;
    d.S = (int32_t)p.S;
    d.t_zhi = p.t_zhi;
    d.t_c64 = p.t_c64;
    d.t_c32 = p.t_c32;
    d.diag_tab64 = p.diag_tab64;
    d.diag_tab32 = p.diag_tab32;
    d.diag_rest = p.diag_rest;
    d.n_diag_rest = p.n_diag_rest;
    return d;
}

template <typename R, int KIND, bool REALH, int TPT, int NBUF>
void launch_one(const ApplyCfg &cfg, const SectorView &v, const Geom &geo, const PlanDev &pd, const void *in,
                void *out, double *partials, int flags, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    auto run = [&](auto kern) {
        smem_optin(reinterpret_cast<const void *>(kern), cfg.smem);
        kern<<<(unsigned)cfg.nct, kThreads, cfg.smem, st>>>(v, geo, pd, static_cast<const C2 *>(in),
                                                             static_cast<C2 *>(out), partials, flags);
        PS_LAUNCH_CHECK();
    };
    if constexpr (KIND == KBLKR) run(k_apply_wide<R, KIND, REALH, TPT, NBUF>);
    else run(k_apply<R, KIND, REALH, TPT, NBUF>);
}

template <typename R, int KIND, bool REALH>
void launch_kind(const ApplyCfg &cfg, const SectorView &v, const Geom &geo, const PlanDev &pd, const void *in,
                 void *out, double *partials, int flags, cudaStream_t st) {
    if (cfg.direct) {
        using C2 = typename Cx<R>::T;
        const C2 *pin = static_cast<const C2 *>(in);
        C2 *pout = static_cast<C2 *>(out);
        const unsigned g = (unsigned)cfg.nct;
        switch (cfg.tpt) {
            case 4: k_apply_direct<R, KIND, REALH, 4><<<g, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
            case 2: k_apply_direct<R, KIND, REALH, 2><<<g, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
            default: k_apply_direct<R, KIND, REALH, 1><<<g, kThreads, 0, st>>>(v, geo, pd, pin, pout, partials, flags); break;
        }
        PS_LAUNCH_CHECK();
        return;
    }
#define PS_L(T, N) launch_one<R, KIND, REALH, T, N>(cfg, v, geo, pd, in, out, partials, flags, st)
    if (cfg.nbuf == 2) {
        switch (cfg.tpt) {
            case 4: PS_L(4, 2); break;
            case 2: PS_L(2, 2); break;
            default: PS_L(1, 2); break;
        }
    } else {
        switch (cfg.tpt) {
            case 8:
                // 8 columns per thread only for rank-staged rows (one or two resident
                // CTAs per SM: more independent gathers per thread instead of more warps)
                if constexpr (KIND == KBLKR) PS_L(8, 1); else PS_L(4, 1);
                break;
            case 4: PS_L(4, 1); break;
            case 2: PS_L(2, 1); break;
            default: PS_L(1, 1); break;
        }
    }
#undef PS_L
}

template <typename R>
void launch_apply_prec(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out,
                       double *partials, void *split_buf, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const Geom geo = make_geom(v, cfg.tpt * kThreads, cfg.nsplit, cfg.split_p0.data(), (int32_t)p.P);
    const PlanDev pd = plan_dev(p);
    const int kind = v.kind == PAULI_SECTOR_FULL ? KFULL
                     : (v.nblk == 1 && cfg.ranked) ? KBLKR
                     : v.irr ? KBLKC
                     : v.nblk == 1 ? KBLK1 : KBLKN;
    void *kout = out;
    int flags = (out ? 1 : 0) | (partials ? 2 : 0);
    if (cfg.nsplit > 1) {
        kout = split_buf;
        flags = 1 | 4;
    }
    if (p.real) {
        if (kind == KFULL) launch_kind<R, KFULL, true>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLK1) launch_kind<R, KBLK1, true>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLKR) launch_kind<R, KBLKR, true>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLKN) launch_kind<R, KBLKN, true>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else launch_kind<R, KBLKC, true>(cfg, v, geo, pd, in, kout, partials, flags, st);
    } else {
        if (kind == KFULL) launch_kind<R, KFULL, false>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLK1) launch_kind<R, KBLK1, false>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLKR) launch_kind<R, KBLKR, false>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else if (kind == KBLKN) launch_kind<R, KBLKN, false>(cfg, v, geo, pd, in, kout, partials, flags, st);
        else launch_kind<R, KBLKC, false>(cfg, v, geo, pd, in, kout, partials, flags, st);
    }
    if (cfg.nsplit > 1) {
        const int cflags = (out ? 1 : 0) | (partials ? 2 : 0);
        k_combine<R><<<(unsigned)cfg.combine_nct, kThreads, 0, st>>>(
            cfg.nsplit, v.dim, static_cast<const C2 *>(split_buf), static_cast<const C2 *>(in), static_cast<C2 *>(out),
            partials, cflags);
        PS_LAUNCH_CHECK();
    }
}

}  // namespace
}  // namespace ps
