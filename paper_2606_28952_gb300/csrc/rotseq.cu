// rotseq.cu -- products of single-group rotations applied tile by tile
// (Trotterised UCCSD / UCCGSD and other product ansatze, Sec. 3.2: the
// "Trotter" column of Table 2).
//
//   psi <- U_{K-1} ... U_1 U_0 psi,   U_k = exp(-i theta_k G_k),
// every G_k Hermitian with one X mask x_k (pauli_rotate's generator).  On a
// single product block the index of t = (t_hi, t_lo) is off + rank(t_hi) D_lo +
// rank(t_lo): a row per high string, a column per low string.  A generator
// whose x_hi is 0 pairs targets inside one row; one whose x_lo is 0 pairs them
// inside one column; any other pairs row t_hi with row t_hi ^ x_hi.  The
// sequence is cut into runs of consecutive generators that share a tile
// shape, each run applied by one launch in which a CTA
//   1. loads its tile of psi into shared memory,
//   2. applies every rotation of the run in order on the tile (a barrier
//      between rotations; each pair {t, t ^ x} is updated by one thread),
//   3. writes the tile back,
// so psi is read and written once per run instead of once per rotation:
//   ROW  runs (x_hi = 0, and diagonal generators): tile = one or more rows;
//   COL  runs (x_lo = 0, and diagonal generators): tile = every row of a
//        block of a few adjacent columns;
//   PAIR runs (one common x_hi != 0, with row-local and diagonal generators):
//        tile = row pairs {r, r ^ x_hi} (or r alone when r ^ x_hi is outside
//        the sector; such rows are skipped when no generator of the run acts
//        inside one row).
// When every generator of a run has tabulated active patterns and keeps the
// sector, the pairs each one rotates are listed at creation and a tile visits
// only those (k_rotseq_list); other runs test every amplitude of the tile
// against every generator (k_rotseq).  Runs whose tile does not fit in shared
// memory (or sectors that are not one product block) fall back to one
// pauli_rotate launch per generator.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {
namespace {

enum : int { RS_ROW = 0, RS_COL = 1, RS_PAIR = 2, RS_EACH = 3 };
constexpr int kSeqThreads = 512;

constexpr int kMaxActive = kActMax;   // active pair patterns kept per generator
constexpr int kGenChunk = 32;         // generator records staged in shared memory at a time
// dynamic shared memory of a tile: 227 KB less the staged records and angles
constexpr size_t kSeqDynMax = 218 * 1024;

struct SeqGen {
    uint64_t x;
    uint64_t m;                 // support S of the active test (np > 0)
    uint64_t zo;                // Z bits common to every term outside S (np > 0)
    uint64_t pat[kMaxActive];   // t & S of every target whose pair rotates (np of them)
    double2 F[kMaxActive];      // f on each active pattern up to the sign (-1)^{zo . s}
    int t0, t1;    // terms of the generator in the sequence's term arrays
    int theta;     // index into the angle array
    int b0;        // lowest set bit of x (-1 for x = 0)
    int np;        // number of active patterns; 0: every pair representative is evaluated
    int l0, l1;    // the generator's entries in the pair lists (list kernels)
    int pad;
    int *status;   // the generator's device status word (sector leaks)
};
static_assert(sizeof(SeqGen) % 8 == 0, "records are staged as 8-byte words");

struct SeqArgs {
    const SeqGen *gens;
    int g0, g1;                 // generators of this run
    const uint64_t *tz;         // [terms] Z masks of the whole sequence
    const double2 *tc;          // [terms] XZ-form coefficients
    const double *theta;        // [K] angles (device)
    uint64_t xh;                // PAIR: the run's common x_hi
    int lw;                     // COL: log2 of the columns per tile
    int has_local;              // PAIR: a generator of the run acts inside one row
};

template <typename R>
__device__ __forceinline__ void phase_sum(const SeqArgs &a, const SeqGen &g, uint64_t s, R &fr, R &fi) {
    for (int k = g.t0; k < g.t1; ++k) {
        const uint32_t par = __popcll(__ldg(a.tz + k) & s);
        const double2 c = __ldg(a.tc + k);
        fr += flip((R)c.x, par);
        fi += flip((R)c.y, par);
    }
}

template <typename R> __device__ __forceinline__ void sincos_s(R a, R *s, R *c);
template <> __device__ __forceinline__ void sincos_s<float>(float a, float *s, float *c) { sincosf(a, s, c); }
template <> __device__ __forceinline__ void sincos_s<double>(double a, double *s, double *c) { sincos(a, s, c); }

// Entry e of a tile: row rs, column cc (ROW: one row; PAIR: two rows of ld
// columns; COL: rows of 2^lw columns).
template <int MODE>
__device__ __forceinline__ void seq_entry(int e, int ld, int lw, int &rs, int &cc) {
    if (MODE == RS_ROW) {
        rs = 0;
        cc = e;
    } else if (MODE == RS_PAIR) {
        rs = e >= ld;
        cc = e - rs * ld;
    } else {
        rs = e >> lw;
        cc = e & ((1 << lw) - 1);
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kSeqThreads, 2)
k_rotseq(SectorView v, SeqArgs A, typename Cx<R>::T *__restrict__ psi) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) char smem[];
    const int tid = threadIdx.x;
    const int klo = v.klo[0], khi = v.khi[0];
    const int64_t dlo = v.dlo[0], off = v.off[0];
    const uint32_t *lst_lo = v.list_lo + v.lst_lo_off[0];
    const uint32_t *lst_hi = v.list_hi + v.lst_hi_off[0];
    const uint64_t lomask = (1ull << v.n_lo) - 1ull;
    int nrow = 1, ld = (int)dlo, ncol = (int)dlo;
    int64_t c0 = 0;
    int64_t rrank[2] = {0, 0};
    uint32_t rpat[2] = {0u, 0u};
    if (MODE == RS_COL) {
        ld = 1 << A.lw;
        c0 = (int64_t)blockIdx.x * ld;
        ncol = (int)min((int64_t)ld, dlo - c0);
        nrow = (int)v.dhi[0];
    } else {
        const int64_t i = blockIdx.x;
        rpat[0] = __ldg(lst_hi + i);
        rrank[0] = i;
        if (MODE == RS_PAIR) {
            const uint32_t r2 = rpat[0] ^ (uint32_t)A.xh;
            if (cls_hi(v, r2) == khi) {
                const int64_t j = __ldg(v.rank_hi + r2);
                if (j < i) return;  // the partner row's block owns this pair of rows
                rpat[1] = r2;
                rrank[1] = j;
                nrow = 2;
            } else if (!A.has_local) {
                return;  // no generator of the run acts on a row whose partner is outside the sector
            }
        }
    }
    C2 *tile = reinterpret_cast<C2 *>(smem);
    uint32_t *tlo_s = reinterpret_cast<uint32_t *>(smem + (size_t)nrow * ld * sizeof(C2));
    uint32_t *thi_s = tlo_s + ld;
    const int nent = nrow * ld;
    // 1. the tile -> shared memory (rows are contiguous runs of ncol amplitudes),
    //    with the strings of its rows and columns
    for (int c = tid; c < ncol; c += kSeqThreads) tlo_s[c] = __ldg(lst_lo + c0 + c);
    for (int r = tid; r < nrow; r += kSeqThreads) thi_s[r] = (MODE == RS_COL) ? __ldg(lst_hi + r) : rpat[r];
    for (int e = tid; e < nent; e += kSeqThreads) {
        int rs, cc;
        seq_entry<MODE>(e, ld, A.lw, rs, cc);
        if (cc >= ncol) continue;
        const int64_t rowrank = (MODE == RS_COL) ? rs : rrank[rs];
        tile[e] = psi[off + rowrank * dlo + c0 + cc];
    }
    __syncthreads();
    // 2. the run's rotations, in order, kGenChunk generator records at a time
    //    staged in shared memory with their angles and, per active pattern,
    //    cos / sin of the pattern's angle; a target is skipped unless its pair
    //    can rotate (its pattern on the generator's support is active)
    __shared__ SeqGen sg[kGenChunk];
    __shared__ R s_th[kGenChunk];
    __shared__ R s_cs[kGenChunk][kMaxActive], s_q[kGenChunk][kMaxActive];
    for (int c0g = A.g0; c0g < A.g1; c0g += kGenChunk) {
        const int nc = min(kGenChunk, A.g1 - c0g);
        {
            const uint64_t *src = reinterpret_cast<const uint64_t *>(A.gens + c0g);
            uint64_t *dst = reinterpret_cast<uint64_t *>(sg);
            for (int wd = tid; wd < nc * (int)(sizeof(SeqGen) / 8); wd += kSeqThreads) dst[wd] = __ldg(src + wd);
        }
        __syncthreads();
        if (tid < nc * kMaxActive) {
            const int gi = tid / kMaxActive, k = tid - gi * kMaxActive;
            const SeqGen &g = sg[gi];
            const double th = __ldg(A.theta + g.theta);
            if (k == 0) s_th[gi] = (R)th;
            double cs = 1.0, q = 0.0;
            if (k < g.np) {
                const double2 F = g.F[k];
                if (g.x == 0) {
                    // diagonal: exp(-i theta f) with f = +-F (real); the sign goes on the sine
                    cs = cos(th * F.x);
                    q = sin(th * F.x);
                } else {
                    const double mag = hypot(F.x, F.y);
                    cs = cos(th * mag);
                    q = sin(th * mag) / mag;
                }
            }
            s_cs[gi][k] = (R)cs;
            s_q[gi][k] = (R)q;
        }
        __syncthreads();
        for (int gi = 0; gi < nc; ++gi) {
            const SeqGen &g = sg[gi];
            const uint64_t gx = g.x, gm = g.m, gzo = g.zo;
            const int np = g.np, b0 = g.b0;
            const R theta = s_th[gi];
            for (int e = tid; e < nent; e += kSeqThreads) {
                int rs, cc;
                seq_entry<MODE>(e, ld, A.lw, rs, cc);
                if (cc >= ncol) continue;
                const uint32_t thi = thi_s[rs], tlo = tlo_s[cc];
                const uint64_t t = (uint64_t)tlo | ((uint64_t)thi << v.n_lo);
                const uint64_t s = t ^ gx;   // the pair partner (t itself for a diagonal generator)
                R fr = R(0), fi = R(0), cs, q;
                if (np != 0) {
                    const uint64_t tm = t & gm;
                    int kk = -1;
#pragma unroll
                    for (int k = 0; k < kMaxActive; ++k)
                        if (k < np && tm == g.pat[k]) kk = k;
                    if (kk < 0) continue;
                    const uint32_t par = __popcll(gzo & s);
                    const double2 F = g.F[kk];
                    fr = flip((R)F.x, par);
                    fi = flip((R)F.y, par);
                    cs = s_cs[gi][kk];
                    q = (gx == 0) ? flip(s_q[gi][kk], par) : s_q[gi][kk];
                } else {
                    if (gx != 0 && !((t >> b0) & 1ull)) continue;  // each pair from its member with bit b0 set
                    phase_sum<R>(A, g, s, fr, fi);
                    if (gx == 0) {
                        sincos_s<R>(theta * fr, &q, &cs);
                    } else {
                        const R mag = sqrt(fr * fr + fi * fi);
                        if (mag == R(0)) {
                            cs = R(1);
                            q = R(0);
                        } else {
                            R sn;
                            sincos_s<R>(theta * mag, &sn, &cs);
                            q = sn / mag;
                        }
                    }
                }
                if (gx == 0) {
                    // exp(-i theta f_t) on one amplitude (f real for a Hermitian diagonal
                    // generator): cs = cos(theta f_t), q = sin(theta f_t)
                    const C2 a = tile[e];
                    C2 o;
                    o.x = cs * a.x + q * a.y;
                    o.y = cs * a.y - q * a.x;
                    tile[e] = o;
                    continue;
                }
                const uint32_t slo = (uint32_t)(s & lomask), shi = (uint32_t)(s >> v.n_lo);
                bool in = cls_lo(v, slo) == klo && cls_hi(v, shi) == khi;
                int pe = 0;
                if (in) {
                    if (MODE == RS_COL) {
                        pe = ((int)__ldg(v.rank_hi + shi) << A.lw) + cc;
                    } else {
                        int prs = rs;
                        if (shi != thi) prs = (nrow == 2 && shi == rpat[rs ^ 1]) ? (rs ^ 1) : -1;
                        if (prs < 0) in = false;
                        else pe = prs * ld + (int)__ldg(v.rank_lo + slo);
                    }
                }
                if (!in) {
                    if (fr != R(0) || fi != R(0)) atomicCAS(g.status, 0, (int)PAULI_ESECTOR);
                    continue;
                }
                if (q == R(0) && cs == R(1)) continue;  // f = 0 (or a zero angle): nothing moves
                const C2 a = tile[e], b = tile[pe];
                const R wr = fr * b.x - fi * b.y, wi = fr * b.y + fi * b.x;   // f b
                const R ur = fr * a.x + fi * a.y, ui = fr * a.y - fi * a.x;   // conj(f) a
                C2 na, nb;
                na.x = cs * a.x + q * wi;
                na.y = cs * a.y - q * wr;
                nb.x = cs * b.x + q * ui;
                nb.y = cs * b.y - q * ur;
                tile[e] = na;
                tile[pe] = nb;
            }
            __syncthreads();
        }
    }
    // 3. the tile -> psi
    for (int e = tid; e < nent; e += kSeqThreads) {
        int rs, cc;
        seq_entry<MODE>(e, ld, A.lw, rs, cc);
        if (cc >= ncol) continue;
        const int64_t rowrank = (MODE == RS_COL) ? rs : rrank[rs];
        psi[off + rowrank * dlo + c0 + cc] = tile[e];
    }
}

// ---------------------------------------------------------------------------
// List kernels.  When every generator of a run has tabulated active patterns
// and keeps the sector, the pairs it rotates are known before the run: a
// ROW or PAIR generator rotates column c with column pc of the same (ROW) or
// the paired (PAIR) row when the row's pattern on S also matches; a COL
// generator rotates row r with row pr of every column whose pattern matches.
// Each generator has a list of entries {index, partner | kk << 24 | sgn << 31}
// (kk: the active pattern, sgn: the parity of z_o on the partner's listed
// half), so a tile visits only the targets that rotate instead of testing
// every amplitude against every generator.
// ---------------------------------------------------------------------------
constexpr int kListThreads = 256;

struct ListArgs {
    const SeqGen *gens;
    int g0, g1;
    const double *theta;   // [K] angles (device)
    const uint2 *lst;      // every generator's entries
    const int2 *pairs;     // PAIR: the run's row pairs (ranks; y = -1: a row without a partner)
    int64_t nunits;        // ROW: rows, COL: columns, PAIR: row pairs
    int per_tile;          // ROW: rows, PAIR: row pairs, COL: 1 << lw columns per tile
    int lw;                // COL: log2 of the columns per tile
};

// it -> (it / L, it % L) for it < 2^24: float quotient, corrected by one step
__device__ __forceinline__ void div_small(int it, int L, float invL, int &qt, int &rm) {
    qt = __float2int_rz((float)it * invL);
    if (qt * L > it) --qt;
    else if ((qt + 1) * L <= it) ++qt;
    rm = it - qt * L;
}

template <typename R>
__device__ __forceinline__ void rotate_pair(typename Cx<R>::T *tile, int ea, int eb, bool diag, R fr, R fi, R cs, R q) {
    using C2 = typename Cx<R>::T;
    if (diag) {
        // exp(-i theta f) on one amplitude: cs = cos(theta f), q = sin(theta f)
        const C2 a = tile[ea];
        C2 o;
        o.x = cs * a.x + q * a.y;
        o.y = cs * a.y - q * a.x;
        tile[ea] = o;
        return;
    }
    const C2 a = tile[ea], b = tile[eb];
    const R wr = fr * b.x - fi * b.y, wi = fr * b.y + fi * b.x;   // f b
    const R ur = fr * a.x + fi * a.y, ui = fr * a.y - fi * a.x;   // conj(f) a
    C2 na, nb;
    na.x = cs * a.x + q * wi;
    na.y = cs * a.y - q * wr;
    nb.x = cs * b.x + q * ui;
    nb.y = cs * b.y - q * ur;
    tile[ea] = na;
    tile[eb] = nb;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(kListThreads)
k_rotseq_list(SectorView v, ListArgs A, typename Cx<R>::T *__restrict__ psi) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) char smem[];
    const int tid = threadIdx.x;
    const int64_t dlo = v.dlo[0], dhi = v.dhi[0], off = v.off[0];
    const uint32_t *lst_lo = v.list_lo + v.lst_lo_off[0];
    const uint32_t *lst_hi = v.list_hi + v.lst_hi_off[0];
    const int n_lo = v.n_lo;
    const int64_t u0 = (int64_t)blockIdx.x * A.per_tile;
    int nrow, ncol, ld, nslot = 0;
    int64_t c0 = 0;
    if (MODE == RS_ROW) {
        nrow = (int)min((int64_t)A.per_tile, dhi - u0);
        ncol = ld = (int)dlo;
    } else if (MODE == RS_PAIR) {
        nslot = (int)min((int64_t)A.per_tile, A.nunits - u0);
        nrow = 2 * nslot;
        ncol = ld = (int)dlo;
    } else {
        ld = 1 << A.lw;
        c0 = u0;
        ncol = (int)min((int64_t)ld, dlo - c0);
        nrow = (int)dhi;
    }
    C2 *tile = reinterpret_cast<C2 *>(smem);
    uint32_t *thi_s = reinterpret_cast<uint32_t *>(smem + (size_t)nrow * ld * sizeof(C2));
    int *rrank = reinterpret_cast<int *>(thi_s + nrow);
    uint32_t *tlo_s = reinterpret_cast<uint32_t *>(rrank + nrow);  // COL: [ld]
    // 1. rows of the tile, then the tile -> shared memory
    for (int r = tid; r < nrow; r += kListThreads) {
        int64_t rk;
        if (MODE == RS_ROW) rk = u0 + r;
        else if (MODE == RS_PAIR) {
            const int2 pr = __ldg(A.pairs + u0 + (r >> 1));
            rk = (r & 1) ? pr.y : pr.x;
        } else rk = r;
        rrank[r] = (int)rk;
        thi_s[r] = rk >= 0 ? __ldg(lst_hi + rk) : 0u;
    }
    if (MODE == RS_COL)
        for (int c = tid; c < ld; c += kListThreads) tlo_s[c] = c < ncol ? __ldg(lst_lo + c0 + c) : 0u;
    __syncthreads();
    const int nent = nrow * ld;
    for (int e = tid; e < nent; e += kListThreads) {
        int r, c;
        if (MODE == RS_COL) {
            r = e >> A.lw;
            c = e & (ld - 1);
        } else {
            r = e / ld;
            c = e - r * ld;
        }
        if (c >= ncol || rrank[r] < 0) continue;
        tile[e] = psi[off + (int64_t)rrank[r] * dlo + c0 + c];
    }
    // 2. the run's rotations in order, records and angles staged per chunk
    __shared__ SeqGen sg[kGenChunk];
    __shared__ R s_cs[kGenChunk][kMaxActive], s_q[kGenChunk][kMaxActive];
    for (int c0g = A.g0; c0g < A.g1; c0g += kGenChunk) {
        const int nc = min(kGenChunk, A.g1 - c0g);
        __syncthreads();
        {
            const uint64_t *src = reinterpret_cast<const uint64_t *>(A.gens + c0g);
            uint64_t *dst = reinterpret_cast<uint64_t *>(sg);
            for (int wd = tid; wd < nc * (int)(sizeof(SeqGen) / 8); wd += kListThreads) dst[wd] = __ldg(src + wd);
        }
        __syncthreads();
        if (tid < nc * kMaxActive) {
            const int gi = tid / kMaxActive, k = tid - gi * kMaxActive;
            const SeqGen &g = sg[gi];
            const double th = __ldg(A.theta + g.theta);
            double cs = 1.0, q = 0.0;
            if (k < g.np) {
                const double2 F = g.F[k];
                if (g.x == 0) {
                    cs = cos(th * F.x);
                    q = sin(th * F.x);
                } else {
                    const double mag = hypot(F.x, F.y);
                    cs = cos(th * mag);
                    q = sin(th * mag) / mag;
                }
            }
            s_cs[gi][k] = (R)cs;
            s_q[gi][k] = (R)q;
        }
        __syncthreads();
        for (int gi = 0; gi < nc; ++gi) {
            const SeqGen &g = sg[gi];
            const int L = g.l1 - g.l0;
            const bool diag = g.x == 0;
            const uint32_t S_hi = (uint32_t)(g.m >> n_lo), zo_hi = (uint32_t)(g.zo >> n_lo);
            const uint32_t S_lo = (uint32_t)(g.m & ((1ull << n_lo) - 1ull));
            const uint32_t zo_lo = (uint32_t)(g.zo & ((1ull << n_lo) - 1ull));
            const bool pairing = MODE == RS_PAIR && (g.x >> n_lo) != 0;
            const int units = (MODE == RS_COL) ? ncol : (pairing ? nslot : nrow);
            const int items = (MODE == RS_COL) ? (L << A.lw) : units * L;
            const float invL = L > 0 ? 1.0f / (float)L : 0.0f;
            for (int it = tid; it < items; it += kListThreads) {
                int u, j;
                if (MODE == RS_COL) {
                    j = it >> A.lw;
                    u = it & (ld - 1);
                    if (u >= ncol) continue;
                } else {
                    div_small(it, L, invL, u, j);
                }
                const uint2 en = __ldg(A.lst + g.l0 + j);
                const int kk = (int)((en.y >> 24) & 3u);
                uint32_t par = en.y >> 31;
                const int pidx = (int)(en.y & 0xFFFFFFu);
                int ea, eb;
                if (MODE == RS_COL) {
                    // rows en.x -> pidx of column u; the column's pattern must match
                    const uint32_t tlo = tlo_s[u];
                    if ((tlo & S_lo) != (uint32_t)(g.pat[kk] & ((1ull << n_lo) - 1ull))) continue;
                    par ^= __popc(zo_lo & tlo) & 1u;
                    ea = ((int)en.x << A.lw) + u;
                    eb = (pidx << A.lw) + u;
                } else if (pairing) {
                    // columns en.x -> pidx across the row pair u; the row holding the target
                    // is the one whose pattern on S matches
                    const int ra = 2 * u, rb = 2 * u + 1;
                    if (rrank[rb] < 0) continue;
                    const uint32_t ph = (uint32_t)(g.pat[kk] >> n_lo);
                    int rt, rs;
                    if ((thi_s[ra] & S_hi) == ph) {
                        rt = ra;
                        rs = rb;
                    } else if ((thi_s[rb] & S_hi) == ph) {
                        rt = rb;
                        rs = ra;
                    } else {
                        continue;
                    }
                    par ^= __popc(zo_hi & thi_s[rs]) & 1u;
                    ea = rt * ld + (int)en.x;
                    eb = rs * ld + pidx;
                } else {
                    // columns en.x -> pidx inside row u; the row's pattern must match
                    if (rrank[u] < 0) continue;
                    const uint32_t thi = thi_s[u];
                    if ((thi & S_hi) != (uint32_t)(g.pat[kk] >> n_lo)) continue;
                    par ^= __popc(zo_hi & thi) & 1u;
                    ea = u * ld + (int)en.x;
                    eb = u * ld + pidx;
                }
                const double2 F = g.F[kk];
                const R cs = s_cs[gi][kk];
                const R q = diag ? flip(s_q[gi][kk], par) : s_q[gi][kk];
                rotate_pair<R>(tile, ea, eb, diag, flip((R)F.x, par), flip((R)F.y, par), cs, q);
            }
            __syncthreads();
        }
    }
    // 3. the tile -> psi
    for (int e = tid; e < nent; e += kListThreads) {
        int r, c;
        if (MODE == RS_COL) {
            r = e >> A.lw;
            c = e & (ld - 1);
        } else {
            r = e / ld;
            c = e - r * ld;
        }
        if (c >= ncol || rrank[r] < 0) continue;
        psi[off + (int64_t)rrank[r] * dlo + c0 + c] = tile[e];
    }
}

}  // namespace
}  // namespace ps

using namespace ps;

struct pauli_rotseq {
    uint32_t magic;
    Allocator al;
    int K = 0;
    const pauli_sector *s = nullptr;   // must outlive the sequence
    std::vector<pauli_sum *> G;        // generators (must outlive the sequence; used by the fallback)
    struct Run {
        int mode;       // RS_ROW / RS_COL / RS_PAIR (fused) or RS_EACH (one pauli_rotate per generator)
        int g0, g1;
        uint64_t xh;
        int has_local;
        int list = 0;        // 1: pair lists built (k_rotseq_list)
        int64_t nunits = 0;  // list kernels: rows (ROW), columns (COL), row pairs (PAIR)
        int64_t pairs0 = 0;  // PAIR: first row pair in d_pairs
    };
    std::vector<Run> runs;
    std::vector<int> rec_theta;        // angle index of each generator record (fallback launches)
    SeqGen *d_gens = nullptr;
    uint64_t *d_tz = nullptr;
    double2 *d_tc = nullptr;
    double *d_theta = nullptr;
    uint2 *d_list = nullptr;   // pair-list entries of every list run's generators
    int2 *d_pairs = nullptr;   // row pairs of the PAIR list runs
};

namespace {
constexpr uint32_t kSeqMagic = 0x50525331u;  // "PRS1"

void free_seq(pauli_rotseq *q) {
    if (!q) return;
    dev_free(q->al, q->d_gens);
    dev_free(q->al, q->d_tz);
    dev_free(q->al, q->d_tc);
    dev_free(q->al, q->d_theta);
    dev_free(q->al, q->d_list);
    dev_free(q->al, q->d_pairs);
    q->magic = 0;
    delete q;
}

// Shared memory of one tile: nrow x ld amplitudes, the low strings of its
// columns (u32 [ld]) and the high strings of its rows (u32 [nrow]).
size_t tile_bytes(int64_t nrow, int64_t ld, size_t es) {
    return (size_t)nrow * (size_t)ld * es + (size_t)ld * 4 + (size_t)nrow * 4;
}

// log2 of the columns of a COL tile: 32-byte row segments, halved while the
// grid would hold fewer than two tiles per SM or the tile does not fit
int col_lw(const SectorView &v, size_t es) {
    int lw = es == 8 ? 2 : 1;
    const int64_t want = 2 * (int64_t)num_sms();
    while (lw > 0 && ((v.dlo[0] + (1ll << lw) - 1) >> lw) < want) --lw;
    while (lw > 0 && tile_bytes(v.dhi[0], 1ll << lw, es) > kSeqDynMax) --lw;
    return lw;
}

}  // namespace

ActivePatterns ps::find_active_patterns(uint64_t x, const uint64_t *z, const double2 *c, int64_t m) {
    ActivePatterns ap;
    if (m <= 0) return ap;
    uint64_t d = 0;
    for (int64_t k = 0; k < m; ++k) d |= z[k] ^ z[0];
    const uint64_t S = x | d;
    if (__builtin_popcountll(S) > 14) return ap;
    const int b0 = x ? __builtin_ctzll(x) : -1;
    std::vector<uint64_t> act;
    std::vector<double2> fval;
    uint64_t q = 0;
    do {
        if (x == 0 || ((q >> b0) & 1ull)) {
            const uint64_t sq = q ^ x;  // the partner's bits on S (x lies inside S)
            double fr = 0.0, fi = 0.0;
            for (int64_t k = 0; k < m; ++k) {
                const bool odd = __builtin_popcountll(z[k] & sq) & 1;
                fr += odd ? -c[k].x : c[k].x;
                fi += odd ? -c[k].y : c[k].y;
            }
            if (fr != 0.0 || fi != 0.0) {
                act.push_back(q);
                fval.push_back(make_double2(fr, fi));
                if ((int)act.size() > kActMax) return ap;
            }
        }
        q = (q - S) & S;  // next subset of S
    } while (q != 0);
    ap.S = S;
    ap.zo = z[0] & ~S;
    ap.np = act.empty() ? -1 : (int)act.size();
    for (size_t k = 0; k < act.size(); ++k) {
        ap.pat[k] = act[k];
        ap.F[k] = fval[k];
    }
    return ap;
}

namespace {

// The rotation-sequence record's copy of the generator's active patterns
// (the per-target sums in term order: the complex128 values are the same bits).
void active_patterns(SeqGen &g, const std::vector<uint64_t> &hz, const std::vector<double2> &hc) {
    const ActivePatterns ap = find_active_patterns(g.x, hz.data(), hc.data(), (int64_t)hz.size());
    g.np = ap.np;
    g.m = ap.S;
    g.zo = ap.zo;
    for (int k = 0; k < kMaxActive; ++k) {
        g.pat[k] = ap.pat[k];
        g.F[k] = ap.F[k];
    }
}

// Tile of a list run: rows (ROW), row pairs (PAIR) or 2^lw columns (COL) per
// CTA, at most ~100 KB so that two CTAs share an SM, and at least two tiles per
// SM where the sector allows; smem = 0 when one unit does not fit.
struct ListTile {
    int per_tile = 1, lw = 0;
    size_t smem = 0;
};
ListTile list_tile(const pauli_rotseq::Run &r, const SectorView &v, size_t es) {
    ListTile t;
    const int64_t want = 2 * (int64_t)num_sms();
    const size_t budget = 100 * 1024;
    const int64_t dlo = v.dlo[0], dhi = v.dhi[0];
    if (r.mode == RS_COL) {
        auto bytes = [&](int lw) { return (size_t)dhi * (((size_t)es << lw) + 8) + ((size_t)4 << lw); };
        int lw = es == 8 ? 2 : 1;
        while (lw > 0 && ((dlo + (1ll << lw) - 1) >> lw) < want) --lw;
        while (lw > 0 && bytes(lw) > budget) --lw;
        t.lw = lw;
        t.per_tile = 1 << lw;
        t.smem = bytes(lw) <= kSeqDynMax ? bytes(lw) : 0;
        return t;
    }
    const size_t unit = (r.mode == RS_PAIR ? 2 : 1) * ((size_t)dlo * es + 8);
    const int64_t fit = (int64_t)(budget / unit);
    const int64_t spread = std::max<int64_t>(1, r.nunits / want);
    t.per_tile = (int)std::max<int64_t>(1, std::min(fit, spread));
    t.smem = (size_t)t.per_tile * unit <= kSeqDynMax ? (size_t)t.per_tile * unit : 0;
    return t;
}

template <typename R>
void launch_run_list(const pauli_rotseq *q, const pauli_rotseq::Run &r, const ListTile &t, void *psi,
                     cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const SectorView &v = q->s->v;
    ListArgs A;
    A.gens = q->d_gens;
    A.g0 = r.g0;
    A.g1 = r.g1;
    A.theta = q->d_theta;
    A.lst = q->d_list;
    A.pairs = q->d_pairs + r.pairs0;
    A.nunits = r.nunits;
    A.per_tile = t.per_tile;
    A.lw = t.lw;
    const int64_t grid = (r.nunits + t.per_tile - 1) / t.per_tile;
    if (grid <= 0) return;
    PS_CHECK(grid < (1ll << 31), PAULI_EUNSUPPORTED, "rotation sequence: too many tiles");
    C2 *p = static_cast<C2 *>(psi);
    auto go = [&](auto kern) {
        smem_optin(reinterpret_cast<const void *>(kern), t.smem);
        kern<<<(unsigned)grid, kListThreads, t.smem, st>>>(v, A, p);
        PS_LAUNCH_CHECK();
    };
    if (r.mode == RS_ROW) go(k_rotseq_list<R, RS_ROW>);
    else if (r.mode == RS_PAIR) go(k_rotseq_list<R, RS_PAIR>);
    else go(k_rotseq_list<R, RS_COL>);
}

// Pair lists of one run (single product block), or false when a generator is
// not tabulated or could leave the sector (the run then keeps the scanning kernel).
struct HostSector {
    int n_lo, n_hi, klo, khi;
    std::vector<uint32_t> lstr, hstr, rk_lo, rk_hi;
};
bool build_run_lists(const SectorView &v, const HostSector &h, pauli_rotseq::Run &run, std::vector<SeqGen> &gens,
                     std::vector<uint2> &lst, std::vector<int2> &pairs) {
    const uint64_t lomask = (1ull << h.n_lo) - 1ull;
    const int64_t dlo = (int64_t)h.lstr.size(), dhi = (int64_t)h.hstr.size();
    if (dlo >= (1 << 24) || dhi >= (1 << 24)) return false;
    for (int gi = run.g0; gi < run.g1; ++gi)
        if (gens[gi].np == 0) return false;
    const size_t lst_start = lst.size(), pairs_start = pairs.size();
    auto fail = [&]() {
        lst.resize(lst_start);
        pairs.resize(pairs_start);
        return false;
    };
    for (int gi = run.g0; gi < run.g1; ++gi) {
        SeqGen &g = gens[gi];
        g.l0 = (int)lst.size();
        if (g.np > 0) {
            const uint32_t xlo = (uint32_t)(g.x & lomask), xhi = (uint32_t)(g.x >> h.n_lo);
            const uint32_t Slo = (uint32_t)(g.m & lomask), Shi = (uint32_t)(g.m >> h.n_lo);
            const uint32_t zlo = (uint32_t)(g.zo & lomask), zhi = (uint32_t)(g.zo >> h.n_lo);
            if (run.mode == RS_COL) {
                for (int64_t rr = 0; rr < dhi; ++rr) {
                    const uint32_t thi = h.hstr[rr];
                    for (int k = 0; k < g.np; ++k) {
                        if ((thi & Shi) != (uint32_t)(g.pat[k] >> h.n_lo)) continue;
                        const uint32_t shi = thi ^ xhi;
                        if (half_cls(shi, v.irr, v.irr_hi) != h.khi) return fail();
                        const uint32_t sg = (uint32_t)(__builtin_popcount(zhi & shi) & 1);
                        lst.push_back(make_uint2((uint32_t)rr, h.rk_hi[shi] | ((uint32_t)k << 24) | (sg << 31)));
                    }
                }
            } else {
                for (int64_t c = 0; c < dlo; ++c) {
                    const uint32_t tlo = h.lstr[c];
                    for (int k = 0; k < g.np; ++k) {
                        if ((tlo & Slo) != (uint32_t)(g.pat[k] & lomask)) continue;
                        const uint32_t slo = tlo ^ xlo;
                        if (half_cls(slo, v.irr, v.irr_lo) != h.klo) return fail();
                        const uint32_t sg = (uint32_t)(__builtin_popcount(zlo & slo) & 1);
                        lst.push_back(make_uint2((uint32_t)c, h.rk_lo[slo] | ((uint32_t)k << 24) | (sg << 31)));
                    }
                }
                if (xhi != 0) {
                    // a pairing generator: every row its patterns select needs its partner row
                    for (int64_t rr = 0; rr < dhi; ++rr)
                        for (int k = 0; k < g.np; ++k)
                            if ((h.hstr[rr] & Shi) == (uint32_t)(g.pat[k] >> h.n_lo) &&
                                half_cls(h.hstr[rr] ^ xhi, v.irr, v.irr_hi) != h.khi)
                                return fail();
                }
            }
        }
        g.l1 = (int)lst.size();
        if (lst.size() >= (size_t)INT_MAX / 2) return fail();
    }
    if (run.mode == RS_ROW) {
        run.nunits = dhi;
    } else if (run.mode == RS_COL) {
        run.nunits = dlo;
    } else {
        run.pairs0 = (int64_t)pairs.size();
        const uint32_t xh = (uint32_t)run.xh;
        for (int64_t i = 0; i < dhi; ++i) {
            const uint32_t p = h.hstr[i] ^ xh;
            if (half_cls(p, v.irr, v.irr_hi) == h.khi) {
                const int64_t j = h.rk_hi[p];
                if (i < j) pairs.push_back(make_int2((int)i, (int)j));
            } else if (run.has_local) {
                pairs.push_back(make_int2((int)i, -1));
            }
        }
        run.nunits = (int64_t)pairs.size() - run.pairs0;
    }
    run.list = 1;
    return true;
}

size_t run_smem(const pauli_rotseq::Run &r, const SectorView &v, size_t es) {
    if (r.mode == RS_ROW) return tile_bytes(1, v.dlo[0], es);
    if (r.mode == RS_PAIR) return tile_bytes(2, v.dlo[0], es);
    return tile_bytes(v.dhi[0], 1ll << col_lw(v, es), es);
}

template <typename R>
void launch_run(const pauli_rotseq *q, const pauli_rotseq::Run &r, void *psi, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const SectorView &v = q->s->v;
    const size_t es = sizeof(C2);
    SeqArgs A;
    A.gens = q->d_gens;
    A.g0 = r.g0;
    A.g1 = r.g1;
    A.tz = q->d_tz;
    A.tc = q->d_tc;
    A.theta = q->d_theta;
    A.xh = r.xh;
    A.lw = col_lw(v, es);
    A.has_local = r.has_local;
    const size_t smem = run_smem(r, v, es);
    C2 *p = static_cast<C2 *>(psi);
    auto go = [&](auto kern, int64_t grid) {
        if (grid <= 0) return;
        PS_CHECK(grid < (1ll << 31), PAULI_EUNSUPPORTED, "rotation sequence: too many tiles");
        smem_optin(reinterpret_cast<const void *>(kern), smem);
        kern<<<(unsigned)grid, kSeqThreads, smem, st>>>(v, A, p);
        PS_LAUNCH_CHECK();
    };
    if (r.mode == RS_ROW) go(k_rotseq<R, RS_ROW>, v.dhi[0]);
    else if (r.mode == RS_PAIR) go(k_rotseq<R, RS_PAIR>, v.dhi[0]);
    else go(k_rotseq<R, RS_COL>, (v.dlo[0] + (1ll << A.lw) - 1) >> A.lw);
}

}  // namespace

extern "C" {

int pauli_rotseq_create(pauli_sum *const *Gs, int K, const pauli_sector *s, pauli_rotseq **out) {
    pauli_rotseq *q = nullptr;
    try {
        clear_error();
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(K >= 1 && K <= (1 << 22), PAULI_EINVAL, "K must be in 1..4194304");
        PS_CHECK(Gs != nullptr, PAULI_EINVAL, "Gs is NULL");
        PS_CHECK(s != nullptr && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        for (int k = 0; k < K; ++k) {
            PS_CHECK(Gs[k] != nullptr && Gs[k]->magic == kSumMagic, PAULI_EINVAL,
                     "sequence: generator " + std::to_string(k) + " is not a valid pauli_sum handle");
            PS_CHECK(Gs[k]->n == s->v.n, PAULI_EINVAL, "sequence: generator and sector qubit counts differ");
            PS_CHECK(Gs[k]->m == 0 || Gs[k]->G == 1, PAULI_EINVAL,
                     "sequence: generator " + std::to_string(k) + " must have exactly one X mask");
            PS_CHECK(Gs[k]->hermitian, PAULI_ENOTHERMITIAN,
                     "sequence: generator " + std::to_string(k) + " is not Hermitian");
        }
        q = new pauli_rotseq();
        q->magic = kSeqMagic;
        q->al = current_allocator();
        q->K = K;
        q->s = s;
        q->G.assign(Gs, Gs + K);
        const SectorView &v = s->v;
        const bool single = v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1;
        // generator records and the terms of every generator (copied from the handles)
        std::vector<SeqGen> gens;
        std::vector<uint64_t> tz;
        std::vector<double2> tc;
        std::vector<int> gen_of;  // sequence position -> record (-1: empty generator)
        for (int k = 0; k < K; ++k) {
            pauli_sum *G = Gs[k];
            if (G->m == 0) {
                gen_of.push_back(-1);
                continue;
            }
            const uint64_t x = group_mask0(G);
            std::vector<uint64_t> hz(G->m);
            std::vector<double2> hc(G->m);
            PS_CUDA(cudaMemcpy(hz.data(), G->z, G->m * 8, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(hc.data(), G->c, G->m * 16, cudaMemcpyDeviceToHost));
            SeqGen g;
            g.x = x;
            g.t0 = (int)tz.size();
            tz.insert(tz.end(), hz.begin(), hz.end());
            tc.insert(tc.end(), hc.begin(), hc.end());
            g.t1 = (int)tz.size();
            g.theta = k;
            g.b0 = x ? __builtin_ctzll(x) : -1;
            g.status = G->status;
            g.pad = 0;
            g.l0 = g.l1 = 0;
            active_patterns(g, hz, hc);
            gen_of.push_back((int)gens.size());
            gens.push_back(g);
        }
        // runs over the records, in sequence order
        const uint64_t lomask = (1ull << v.n_lo) - 1ull;
        pauli_rotseq::Run cur{-1, 0, 0, 0, 0};
        auto flush = [&]() {
            if (cur.mode >= 0 && cur.g1 > cur.g0) q->runs.push_back(cur);
        };
        for (int r = 0; r < (int)gens.size(); ++r) {
            const uint64_t x = gens[r].x, xl = x & lomask, xhh = x >> v.n_lo;
            if (!single) {
                if (cur.mode != RS_EACH) {
                    flush();
                    cur = {RS_EACH, r, r, 0, 0};
                }
                cur.g1 = r + 1;
                continue;
            }
            int mode;
            if (x == 0) mode = cur.mode >= 0 && cur.mode != RS_EACH ? cur.mode : RS_ROW;  // joins any run
            else if (xhh == 0) mode = (cur.mode == RS_PAIR) ? RS_PAIR : RS_ROW;
            else if (xl == 0) mode = RS_COL;
            else mode = RS_PAIR;
            const bool local = x == 0 || xhh == 0;
            bool joins = false;
            if (cur.mode == mode && mode != RS_PAIR) joins = true;
            if (mode == RS_PAIR && cur.mode == RS_PAIR && (xhh == 0 || xhh == cur.xh || x == 0)) joins = true;
            if (mode == RS_PAIR && cur.mode == RS_ROW && xhh != 0) {
                // a row run becomes a row-pair run: its generators act inside each row of the pair
                cur.mode = RS_PAIR;
                cur.xh = xhh;
                cur.has_local = 1;
                joins = true;
            }
            if (!joins) {
                flush();
                cur = {mode, r, r, mode == RS_PAIR ? xhh : 0, 0};
            }
            if (cur.mode == RS_PAIR && local) cur.has_local = 1;
            cur.g1 = r + 1;
        }
        flush();
        // pair lists for the fused runs (single block with rank tables of at most 2^20 entries)
        std::vector<uint2> lst;
        std::vector<int2> pairs;
        if (single && v.n_lo <= 20 && v.n_hi <= 20) {
            HostSector h;
            h.n_lo = v.n_lo;
            h.n_hi = v.n_hi;
            h.klo = v.klo[0];
            h.khi = v.khi[0];
            h.lstr.resize(v.dlo[0]);
            h.hstr.resize(v.dhi[0]);
            h.rk_lo.resize(1ull << v.n_lo);
            h.rk_hi.resize(1ull << v.n_hi);
            PS_CUDA(cudaMemcpy(h.lstr.data(), v.list_lo + v.lst_lo_off[0], v.dlo[0] * 4, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(h.hstr.data(), v.list_hi + v.lst_hi_off[0], v.dhi[0] * 4, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(h.rk_lo.data(), v.rank_lo, (1ull << v.n_lo) * 4, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(h.rk_hi.data(), v.rank_hi, (1ull << v.n_hi) * 4, cudaMemcpyDeviceToHost));
            for (auto &run : q->runs)
                if (run.mode != RS_EACH) build_run_lists(v, h, run, gens, lst, pairs);
        }
        for (const SeqGen &g : gens) q->rec_theta.push_back(g.theta);
        // device copies
        q->d_gens = static_cast<SeqGen *>(dev_alloc(q->al, std::max<size_t>(1, gens.size()) * sizeof(SeqGen)));
        q->d_tz = static_cast<uint64_t *>(dev_alloc(q->al, std::max<size_t>(1, tz.size()) * 8));
        q->d_tc = static_cast<double2 *>(dev_alloc(q->al, std::max<size_t>(1, tc.size()) * 16));
        q->d_theta = static_cast<double *>(dev_alloc(q->al, (size_t)K * sizeof(double)));
        if (!gens.empty()) PS_CUDA(cudaMemcpy(q->d_gens, gens.data(), gens.size() * sizeof(SeqGen), cudaMemcpyHostToDevice));
        if (!tz.empty()) {
            PS_CUDA(cudaMemcpy(q->d_tz, tz.data(), tz.size() * 8, cudaMemcpyHostToDevice));
            PS_CUDA(cudaMemcpy(q->d_tc, tc.data(), tc.size() * 16, cudaMemcpyHostToDevice));
        }
        q->d_list = static_cast<uint2 *>(dev_alloc(q->al, std::max<size_t>(1, lst.size()) * sizeof(uint2)));
        q->d_pairs = static_cast<int2 *>(dev_alloc(q->al, std::max<size_t>(1, pairs.size()) * sizeof(int2)));
        if (!lst.empty()) PS_CUDA(cudaMemcpy(q->d_list, lst.data(), lst.size() * sizeof(uint2), cudaMemcpyHostToDevice));
        if (!pairs.empty())
            PS_CUDA(cudaMemcpy(q->d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice));
        // the generator of each record, for the fallback launches
        q->G.clear();
        for (int k = 0; k < K; ++k)
            if (gen_of[k] >= 0) q->G.push_back(Gs[k]);
        *out = q;
        return PAULI_OK;
    } catch (const Error &e) {
        free_seq(q);
        set_error(e.msg);
        return e.code;
    } catch (...) {
        free_seq(q);
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_rotseq_info(const pauli_rotseq *q, int dtype, int *launches, int *fused) {
    try {
        clear_error();
        PS_CHECK(q && q->magic == kSeqMagic, PAULI_EINVAL, "not a valid pauli_rotseq handle");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        const size_t es = dtype == PAULI_C64 ? 8 : 16;
        int nl = 0, nf = 0;
        for (const auto &r : q->runs) {
            const bool fused = r.mode != RS_EACH && ((r.list && list_tile(r, q->s->v, es).smem > 0) ||
                                                     run_smem(r, q->s->v, es) <= kSeqDynMax);
            if (fused) {
                ++nl;
                nf += r.g1 - r.g0;
            } else {
                nl += r.g1 - r.g0;
            }
        }
        if (launches) *launches = nl;
        if (fused) *fused = nf;
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int pauli_rotseq_apply(pauli_rotseq *q, const double *thetas, void *psi, int dtype, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(q && q->magic == kSeqMagic, PAULI_EINVAL, "not a valid pauli_rotseq handle");
        PS_CHECK(q->s->magic == kSectorMagic, PAULI_EINVAL, "the sequence's sector has been destroyed");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(thetas != nullptr, PAULI_EINVAL, "thetas is NULL");
        PS_CHECK(psi && ((uintptr_t)psi % 16) == 0, PAULI_EINVAL, "psi is NULL or not 16-byte aligned");
        for (int k = 0; k < q->K; ++k) PS_CHECK(std::isfinite(thetas[k]), PAULI_EINVAL, "thetas must be finite");
        cudaStream_t cs = (cudaStream_t)st;
        // the angles: one host-to-device copy into the handle (calls with one handle
        // must be ordered; the copy is staged before this call returns)
        PS_CUDA(cudaMemcpyAsync(q->d_theta, thetas, (size_t)q->K * sizeof(double), cudaMemcpyHostToDevice, cs));
        const size_t es = dtype == PAULI_C64 ? 8 : 16;
        for (const auto &run : q->runs) {
            if (run.mode != RS_EACH && run.list) {
                const ListTile t = list_tile(run, q->s->v, es);
                if (t.smem > 0) {
                    if (dtype == PAULI_C64) launch_run_list<float>(q, run, t, psi, cs);
                    else launch_run_list<double>(q, run, t, psi, cs);
                    continue;
                }
            }
            if (run.mode != RS_EACH && run_smem(run, q->s->v, es) <= kSeqDynMax) {
                if (dtype == PAULI_C64) launch_run<float>(q, run, psi, cs);
                else launch_run<double>(q, run, psi, cs);
                continue;
            }
            // records keep the sequence order of the non-empty generators
            for (int r = run.g0; r < run.g1; ++r) launch_rotate(q->G[r], q->s, thetas[q->rec_theta[r]], psi, dtype, cs);
        }
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_rotseq_destroy(pauli_rotseq *q) {
    if (!q) return PAULI_OK;
    if (q->magic != kSeqMagic) {
        set_error("not a valid pauli_rotseq handle");
        return PAULI_EINVAL;
    }
    clear_error();
    free_seq(q);
    return PAULI_OK;
}

}  // extern "C"
