// svd.cu -- the gather of eq. svd_sreverse_sum: each group's phase sum
// factorised into alpha and beta parts by a singular value decomposition of
// its coefficient matrix (Sec. 2.4, eq. svd_weights / precomp_alpha /
// precomp_beta / dot_product, Algorithm 2), for real operators on a single
// product block.
//
// For group g (X mask x = (x_lo, x_hi)) with the distinct low Z masks
// {Za_mu} and high Z masks {Zb_nu} of its terms, M_{mu nu} = sum of the C_k
// with z_k = (Za_mu, Zb_nu).  M = U S V^T (one-sided Jacobi in FP64, ranks
// with sigma > 1e-12 kept), Wa = U sqrt(S), Wb = V sqrt(S), and
//   f_g(t) = sum_k Fa_g(t_lo, k) Fb_g(t_hi, k),
//   Fa_g(t_lo, k) = sum_mu Wa_{mu k} (-1)^popcount((t_lo ^ x_lo) & Za_mu),
//   Fb_g(t_hi, k) = sum_nu Wb_{nu k} (-1)^popcount((t_hi ^ x_hi) & Zb_nu).
// GPU layout: a CTA owns one row (t_hi, the beta string) and a tile of its
// columns, so Fb_g is one number per (row, group, k), computed by the CTA when
// it stages the group's source row; Fa_g depends on the column only and is
// tabulated by k_svd_fa for a batch of groups at a time (the paper's
// on-the-fly batches: the table of one batch is built, consumed by the
// gather, and overwritten by the next batch; its size is bounded by
// kSvdBatchBytes).  Per (target, group) the gather then needs R_g table
// loads (coalesced along the row) and FMAs: no parity evaluations.  The x = 0
// group (rank n_orb + 2 for a molecule) is tabulated and contracted in FP64
// on the complex64 path as well, as the other gathers treat it.  Batches after
// the first add to the output in a fixed order; the last emits the FP64
// expectation partials.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {

constexpr int kSvdPieceGroups = 64;     // groups per piece (one staged source row)
constexpr int kSvdPieceRanks = 256;     // sum of R_g over a piece
constexpr int kSvdMaxRank = 64;         // largest R_g handled
constexpr size_t kSvdBatchBytes = 256ull << 20;  // Fa table of one on-the-fly batch

struct SvdGroup {
    uint32_t x_lo, x_hi;
    int R, na, nb;         // rank, distinct low / high Z masks
    int za_off, zb_off;    // first mask of the group in za / zb
    int64_t wa_off, wb_off;  // Wa[mu][k] = wa[wa_off + mu * R + k], Wb likewise
    int64_t fa_row;        // first Fa row of the group (global numbering; a batch subtracts its first row)
    int diag;              // x = 0 group: FP64 table and contraction on every path
    int pad;
};

struct SvdPlan {
    int n_lo = 0, klo = -1;
    int64_t dlo = 0;
    int64_t G = 0, fa_rows = 0, diag_rows = 0;
    std::vector<SvdGroup> h_groups;
    std::vector<int> h_pc_g0;          // pieces: [h_pc_g0[q], h_pc_g0[q+1]) groups
    std::vector<int> h_batch_pc0;      // batches: [h_batch_pc0[b], h_batch_pc0[b+1]) pieces
    std::vector<int> h_rank_hist;      // R -> number of groups
    SvdGroup *groups = nullptr;
    int32_t *pc_g0 = nullptr;
    uint32_t *za = nullptr, *zb = nullptr;
    double *wa = nullptr, *wb = nullptr;
    int32_t *fa_g = nullptr, *fa_k = nullptr;   // Fa row -> (group, k)
    void *fa = nullptr;                          // Fa table of one batch ([rows][dlo], R precision)
    int64_t fa_cap_bytes = 0;
    double *fa_diag = nullptr;                   // [R_0][dlo] FP64 table of the x = 0 group
    Allocator al;
};

namespace {

// One-sided Jacobi SVD of a real m x n matrix a (row-major): on return
// a = U S V^T with s[j] = ||column j|| and u (m x n), v (n x n) row-major.
void jacobi_svd(int m, int n, std::vector<double> a, std::vector<double> &u, std::vector<double> &s,
                std::vector<double> &v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < m; ++i) {
                    const double x = a[(size_t)i * n + p], y = a[(size_t)i * n + q];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
                off = std::max(off, std::fabs(ga) / std::sqrt(al * be));
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < m; ++i) {
                    const double x = a[(size_t)i * n + p], y = a[(size_t)i * n + q];
                    a[(size_t)i * n + p] = c * x - sn * y;
                    a[(size_t)i * n + q] = sn * x + c * y;
                }
                for (int i = 0; i < n; ++i) {
                    const double x = v[(size_t)i * n + p], y = v[(size_t)i * n + q];
                    v[(size_t)i * n + p] = c * x - sn * y;
                    v[(size_t)i * n + q] = sn * x + c * y;
                }
            }
        if (off <= 1e-15) break;
    }
    s.assign(n, 0.0);
    u.assign((size_t)m * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double nn = 0.0;
        for (int i = 0; i < m; ++i) nn += a[(size_t)i * n + j] * a[(size_t)i * n + j];
        s[j] = std::sqrt(nn);
        if (s[j] > 0)
            for (int i = 0; i < m; ++i) u[(size_t)i * n + j] = a[(size_t)i * n + j] / s[j];
    }
}

struct SvdDev {
    const SvdGroup *groups;
    const int32_t *pc_g0;
    const uint32_t *za, *zb;
    const double *wa, *wb;
    const int32_t *fa_g, *fa_k;
    double *fa_diag;
};

// Fa rows [row0, row1) of the current batch (and the FP64 rows of the x = 0
// group, when it is in the batch): one thread per (row, column).
template <typename R>
__global__ void k_svd_fa(SvdDev d, int64_t row0, int64_t row1, int64_t dlo, const uint32_t *__restrict__ lst_lo,
                         R *__restrict__ fa) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nrow = row1 - row0;
    if (i >= nrow * dlo) return;
    const int64_t r = i / dlo, c = i - r * dlo;
    const int g = __ldg(d.fa_g + row0 + r), k = __ldg(d.fa_k + row0 + r);
    const SvdGroup G = d.groups[g];
    const uint32_t s = __ldg(lst_lo + c) ^ G.x_lo;
    double val = 0.0;
    for (int mu = 0; mu < G.na; ++mu) {
        const double w = __ldg(d.wa + G.wa_off + (int64_t)mu * G.R + k);
        val += (__popc(s & __ldg(d.za + G.za_off + mu)) & 1) ? -w : w;
    }
    fa[r * dlo + c] = (R)val;
    if (G.diag) d.fa_diag[(int64_t)k * dlo + c] = val;
}

template <typename R, int TPT>
__global__ void __launch_bounds__(kThreads)
k_apply_svd(SectorView v, Geom geo, SvdDev d, int pc0, int pc1, int64_t fa_row0, const R *__restrict__ fa,
            const typename Cx<R>::T *__restrict__ psi, typename Cx<R>::T *__restrict__ out,
            double *__restrict__ partials, int flags) {
    using C2 = typename Cx<R>::T;
    extern __shared__ __align__(16) char smem[];
    const int64_t dlo = v.dlo[0];
    const int klo = v.klo[0], khi = v.khi[0];
    const int rw = ranked_rowcap(dlo);
    C2 *row = reinterpret_cast<C2 *>(smem);
    char *tab = smem + (size_t)rw * sizeof(C2);
    double *fb64 = reinterpret_cast<double *>(tab + ((rank_table_bytes(v.n_lo) + 15) & ~(size_t)15));
    R *fb = reinterpret_cast<R *>(fb64 + kSvdMaxRank);
    int4 *grec = reinterpret_cast<int4 *>(fb + kSvdPieceRanks + 4);  // {x_lo, R, fb offset, diag}
    int64_t *gfa = reinterpret_cast<int64_t *>(grec + kSvdPieceGroups);
    const RowCtx rc = decode_row<false>(v, geo, blockIdx.x);
    const int tid = threadIdx.x;
    // rank table of the low half (as for rank-staged rows)
    RankTab rt;
    rt.lut = reinterpret_cast<const uint16_t *>(tab);
    rt.tabA = reinterpret_cast<const uint32_t *>(tab);
    rt.tabB = rt.tabA + 256;
    rt.n_lo = v.n_lo;
    rt.klo = klo;
    rt.dlo = (uint32_t)dlo;
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
    if (tid == 0) {
        C2 zz;
        zz.x = R(0);
        zz.y = R(0);
        row[dlo] = zz;  // the zero slot of sources outside the block
    }
    uint32_t tlo[TPT];
    int64_t col[TPT];
    bool act[TPT];
    R accr[TPT], acci[TPT];
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        col[j] = rc.c0 + tid + j * kThreads;
        act[j] = col[j] < rc.dlo;
        tlo[j] = act[j] ? __ldg(v.list_lo + v.lst_lo_off[0] + col[j]) : 0u;
        accr[j] = R(0);
        acci[j] = R(0);
    }
    __syncthreads();
    for (int q = pc0; q < pc1; ++q) {
        const int g0 = __ldg(d.pc_g0 + q), g1 = __ldg(d.pc_g0 + q + 1);
        const uint32_t shi = rc.thi ^ d.groups[g0].x_hi;
        if (cls_hi(v, shi) != khi) continue;  // the source row is outside the sector (block-uniform)
        const int64_t base = v.off[0] + (int64_t)__ldg(v.rank_hi + shi) * dlo;
        for (int64_t r = tid; r < dlo; r += kThreads) {
            if (sizeof(C2) == 16) cp_async16(row + r, psi + base + r);
            else cp_async8(row + r, psi + base + r);
        }
        cp_async_commit();
        // group records and the beta factors Fb_g(t_hi, k) of this row (FP64 sums)
        if (tid < g1 - g0) {
            const SvdGroup G = d.groups[g0 + tid];
            int off = 0;
            for (int g = g0; g < g0 + tid; ++g) off += d.groups[g].R;
            grec[tid] = make_int4((int)G.x_lo, G.R, off, G.diag);
            gfa[tid] = G.fa_row - fa_row0;
        }
        __syncthreads();
        for (int e = tid; e < kSvdPieceRanks; e += kThreads) {
            // (group, k) of entry e: walk the piece's records
            int gi = 0, acc_r = 0;
            while (gi < g1 - g0 && acc_r + grec[gi].y <= e) {
                acc_r += grec[gi].y;
                ++gi;
            }
            if (gi >= g1 - g0) break;
            const int k = e - acc_r;
            const SvdGroup G = d.groups[g0 + gi];
            double val = 0.0;
            for (int nu = 0; nu < G.nb; ++nu) {
                const double w = __ldg(d.wb + G.wb_off + (int64_t)nu * G.R + k);
                val += (__popc(shi & __ldg(d.zb + G.zb_off + nu)) & 1) ? -w : w;
            }
            fb[e] = (R)val;
            if (G.diag) fb64[k] = val;
        }
        cp_async_wait<0>();
        __syncthreads();
        for (int gi = 0; gi < g1 - g0; ++gi) {
            const int4 gr = grec[gi];
            const R *fag = fa + gfa[gi] * dlo;
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
                const uint32_t s = tlo[j] ^ (uint32_t)gr.x;
                if (!act[j] || cls_lo(v, s) != klo) continue;  // source outside the block
                const C2 amp = row[ranked_index(rt, s)];
                if (sizeof(R) == 4 && gr.w) {
                    // x = 0 group on the FP32 path: FP64 contraction, applied as hi + lo parts
                    double f = 0.0;
                    for (int k = 0; k < gr.y; ++k) f += d.fa_diag[(int64_t)k * dlo + col[j]] * fb64[k];
                    const R fh = (R)f, fl = (R)(f - (double)fh);
                    accr[j] += fh * amp.x + fl * amp.x;
                    acci[j] += fh * amp.y + fl * amp.y;
                } else {
                    R f = R(0);
                    for (int k = 0; k < gr.y; ++k) f += __ldg(fag + (int64_t)k * dlo + col[j]) * fb[gr.z + k];
                    accr[j] += f * amp.x;
                    acci[j] += f * amp.y;
                }
            }
        }
        __syncthreads();
    }
    // epilogue: store, or add to the earlier batches' sums; FP64 partials
    ExpAcc<R> ea;
#pragma unroll
    for (int j = 0; j < TPT; ++j) {
        if (!act[j]) continue;
        const int64_t idx = rc.own_base + col[j];
        C2 o;
        o.x = accr[j];
        o.y = acci[j];
        if (flags & 8) {
            const C2 p = out[idx];
            o.x = p.x + o.x;
            o.y = p.y + o.y;
        }
        if (flags & 1) out[idx] = o;
        if (flags & 2) ea.add(psi[idx], o.x, o.y);
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

}  // namespace

size_t svd_smem(const SectorView &v, int dtype) {
    const size_t es = dtype == PAULI_C64 ? 8 : 16, rs = dtype == PAULI_C64 ? 4 : 8;
    return (size_t)ranked_rowcap(v.dlo[0]) * es + ((rank_table_bytes(v.n_lo) + 15) & ~(size_t)15) +
           kSvdMaxRank * 8 + (kSvdPieceRanks + 4) * rs + kSvdPieceGroups * (16 + 8) + 64;
}

void free_svd_plan(SvdPlan *sp) {
    if (!sp) return;
    const Allocator &al = sp->al;
    dev_free(al, sp->groups);
    dev_free(al, sp->pc_g0);
    dev_free(al, sp->za);
    dev_free(al, sp->zb);
    dev_free(al, sp->wa);
    dev_free(al, sp->wb);
    dev_free(al, sp->fa_g);
    dev_free(al, sp->fa_k);
    dev_free(al, sp->fa);
    dev_free(al, sp->fa_diag);
    delete sp;
}

// The SVD plan of a real operator on a single-block sector (nullptr if the
// operator is complex, a rank exceeds kSvdMaxRank or the low half is wider
// than 16 qubits).  Blocking.
SvdPlan *build_svd_plan(pauli_sum *H, const SectorView &v, cudaStream_t st) {
    if (!(v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1) || !H->real || H->m == 0 || v.n_lo > (v.irr ? 14 : 16))
        return nullptr;
    const int64_t M = H->m, G = H->G;
    std::vector<uint64_t> z(M), gx(G);
    std::vector<double2> c(M);
    std::vector<int64_t> gs(G + 1);
    PS_CUDA(cudaMemcpyAsync(z.data(), H->z, M * 8, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(c.data(), H->c, M * 16, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(gx.data(), H->gx, G * 8, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(gs.data(), H->gstart, (G + 1) * 8, cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    const uint64_t lomask = (1ull << v.n_lo) - 1ull;
    std::vector<SvdGroup> groups;
    std::vector<uint32_t> za, zb;
    std::vector<double> wa, wb;
    std::vector<int32_t> fa_g, fa_k;
    std::vector<int> hist(kSvdMaxRank + 1, 0);
    int64_t diag_rank = 0;
    for (int64_t g = 0; g < G; ++g) {
        // distinct low / high Z masks of the group's terms; M_{mu nu} = sum of their C
        std::map<uint32_t, int> ia, ib;
        for (int64_t t = gs[g]; t < gs[g + 1]; ++t) {
            ia.emplace((uint32_t)(z[t] & lomask), 0);
            ib.emplace((uint32_t)(z[t] >> v.n_lo), 0);
        }
        int na = 0, nb = 0;
        for (auto &e : ia) e.second = na++;
        for (auto &e : ib) e.second = nb++;
        std::vector<double> Mg((size_t)na * nb, 0.0);
        for (int64_t t = gs[g]; t < gs[g + 1]; ++t)
            Mg[(size_t)ia[(uint32_t)(z[t] & lomask)] * nb + ib[(uint32_t)(z[t] >> v.n_lo)]] += c[t].x;
        double mmax = 0.0;
        for (double e : Mg) mmax = std::max(mmax, std::fabs(e));
        std::vector<double> u, sv, vv;
        jacobi_svd(na, nb, Mg, u, sv, vv);
        std::vector<int> keep;
        for (int j = 0; j < nb; ++j)
            if (sv[j] > 1e-12) keep.push_back(j);  // the paper's truncation sigma_r > 1e-12
        std::sort(keep.begin(), keep.end(), [&](int a, int b) { return sv[a] > sv[b]; });
        const int R = (int)keep.size();
        if (R > kSvdMaxRank) return nullptr;
        ++hist[R];
        // self-check of the factorisation: sum_k Wa Wb^T reproduces M
        for (int a = 0; a < na; ++a)
            for (int b = 0; b < nb; ++b) {
                double r = 0.0;
                for (int j : keep) r += u[(size_t)a * nb + j] * sv[j] * vv[(size_t)b * nb + j];
                PS_CHECK(std::fabs(r - Mg[(size_t)a * nb + b]) <= 1e-10 * std::max(1.0, mmax), PAULI_ECUDA,
                         "svd plan: the factorisation of a group's coefficient matrix did not converge");
            }
        if (R == 0) continue;  // every coefficient of the group cancels
        SvdGroup rec;
        rec.x_lo = (uint32_t)(gx[g] & lomask);
        rec.x_hi = (uint32_t)(gx[g] >> v.n_lo);
        rec.R = R;
        rec.na = na;
        rec.nb = nb;
        rec.za_off = (int)za.size();
        rec.zb_off = (int)zb.size();
        rec.wa_off = (int64_t)wa.size();
        rec.wb_off = (int64_t)wb.size();
        rec.fa_row = (int64_t)fa_g.size();
        rec.diag = gx[g] == 0 ? 1 : 0;
        rec.pad = 0;
        if (rec.diag) diag_rank = R;
        for (auto &e : ia) za.push_back(e.first);
        for (auto &e : ib) zb.push_back(e.first);
        for (int a = 0; a < na; ++a)
            for (int k = 0; k < R; ++k) wa.push_back(u[(size_t)a * nb + keep[k]] * std::sqrt(sv[keep[k]]));
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < R; ++k) wb.push_back(vv[(size_t)b * nb + keep[k]] * std::sqrt(sv[keep[k]]));
        for (int k = 0; k < R; ++k) {
            fa_g.push_back((int32_t)groups.size());
            fa_k.push_back(k);
        }
        groups.push_back(rec);
    }
    auto sp = new SvdPlan();
    sp->al = H->al;
    sp->n_lo = v.n_lo;
    sp->klo = v.klo[0];
    sp->dlo = v.dlo[0];
    sp->G = (int64_t)groups.size();
    sp->fa_rows = (int64_t)fa_g.size();
    sp->diag_rows = diag_rank;
    sp->h_rank_hist = hist;
    sp->h_groups = groups;
    // pieces: runs of groups with one x_hi (one staged source row), bounded in groups and ranks
    sp->h_pc_g0.push_back(0);
    for (int g = 0, cnt = 0, rsum = 0; g < (int)groups.size(); ++g) {
        const bool same = g > 0 && groups[g].x_hi == groups[g - 1].x_hi;
        if (g > 0 && (!same || cnt == kSvdPieceGroups || rsum + groups[g].R > kSvdPieceRanks)) {
            sp->h_pc_g0.push_back(g);
            cnt = 0;
            rsum = 0;
        }
        ++cnt;
        rsum += groups[g].R;
    }
    sp->h_pc_g0.push_back((int)groups.size());
    if (groups.empty()) sp->h_pc_g0.assign(1, 0);
    // on-the-fly batches: ranges of pieces whose Fa rows fit in kSvdBatchBytes (FP64)
    const int P = (int)sp->h_pc_g0.size() - 1;
    sp->h_batch_pc0.push_back(0);
    int64_t rows = 0, max_rows = 0;
    for (int q = 0; q < P; ++q) {
        int64_t r = 0;
        for (int g = sp->h_pc_g0[q]; g < sp->h_pc_g0[q + 1]; ++g) r += groups[g].R;
        if (rows > 0 && (rows + r) * sp->dlo * 8 > (int64_t)kSvdBatchBytes) {
            sp->h_batch_pc0.push_back(q);
            max_rows = std::max(max_rows, rows);
            rows = 0;
        }
        rows += r;
    }
    max_rows = std::max(max_rows, rows);
    sp->h_batch_pc0.push_back(P);
    try {
        auto up = [&](const void *src, size_t bytes) {
            void *d = dev_alloc(sp->al, bytes > 0 ? bytes : 16);
            if (bytes > 0) PS_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
            return d;
        };
        sp->groups = static_cast<SvdGroup *>(up(groups.data(), groups.size() * sizeof(SvdGroup)));
        std::vector<int32_t> pc(sp->h_pc_g0.begin(), sp->h_pc_g0.end());
        sp->pc_g0 = static_cast<int32_t *>(up(pc.data(), pc.size() * sizeof(int32_t)));
        sp->za = static_cast<uint32_t *>(up(za.data(), za.size() * 4));
        sp->zb = static_cast<uint32_t *>(up(zb.data(), zb.size() * 4));
        sp->wa = static_cast<double *>(up(wa.data(), wa.size() * 8));
        sp->wb = static_cast<double *>(up(wb.data(), wb.size() * 8));
        sp->fa_g = static_cast<int32_t *>(up(fa_g.data(), fa_g.size() * 4));
        sp->fa_k = static_cast<int32_t *>(up(fa_k.data(), fa_k.size() * 4));
        sp->fa_cap_bytes = std::max<int64_t>(1, max_rows) * sp->dlo * 8;
        sp->fa = dev_alloc(sp->al, (size_t)sp->fa_cap_bytes);
        sp->fa_diag = static_cast<double *>(dev_alloc(sp->al, (size_t)std::max<int64_t>(1, diag_rank) * sp->dlo * 8));
        PS_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
        free_svd_plan(sp);
        throw;
    }
    return sp;
}

bool svd_plan_fits(const SvdPlan *sp, const SectorView &v) {
    return sp && v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1 && sp->n_lo == v.n_lo && sp->klo == v.klo[0] &&
           sp->dlo == v.dlo[0];
}

int svd_batches(const SvdPlan *sp) { return sp ? (int)sp->h_batch_pc0.size() - 1 : 0; }

const std::vector<int> &svd_rank_hist(const SvdPlan *sp) { return sp->h_rank_hist; }

template <typename R, int TPT>
static void launch_svd_t(const ApplyCfg &cfg, const SvdPlan &sp, const SectorView &v, const void *in, void *out,
                         double *partials, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    const Geom geo = make_geom(v, TPT * kThreads);
    SvdDev d;
    d.groups = sp.groups;
    d.pc_g0 = sp.pc_g0;
    d.za = sp.za;
    d.zb = sp.zb;
    d.wa = sp.wa;
    d.wb = sp.wb;
    d.fa_g = sp.fa_g;
    d.fa_k = sp.fa_k;
    d.fa_diag = sp.fa_diag;
    const uint32_t *lst_lo = v.list_lo + v.lst_lo_off[0];
    const int nb = (int)sp.h_batch_pc0.size() - 1;
    const size_t smem = cfg.smem;
    auto kern = k_apply_svd<R, TPT>;
    smem_optin(reinterpret_cast<const void *>(kern), smem);
    for (int b = 0; b < nb; ++b) {
        const int pc0 = sp.h_batch_pc0[b], pc1 = sp.h_batch_pc0[b + 1];
        const int g0 = sp.h_pc_g0[pc0], g1 = sp.h_pc_g0[pc1];
        const int64_t row0 = g0 < (int)sp.h_groups.size() ? sp.h_groups[g0].fa_row : sp.fa_rows;
        const int64_t row1 = g1 < (int)sp.h_groups.size() ? sp.h_groups[g1].fa_row : sp.fa_rows;
        const int64_t n = (row1 - row0) * sp.dlo;
        if (n > 0) {
            k_svd_fa<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, row0, row1, sp.dlo, lst_lo,
                                                                     static_cast<R *>(sp.fa));
            PS_LAUNCH_CHECK();
        }
        const int flags = (out ? 1 : 0) | (b > 0 ? 8 : 0) | ((b == nb - 1 && partials) ? 2 : 0);
        void *o = out;
        kern<<<(unsigned)cfg.nct, kThreads, smem, st>>>(v, geo, d, pc0, pc1, row0, static_cast<const R *>(sp.fa),
                                                        static_cast<const C2 *>(in), static_cast<C2 *>(o), partials,
                                                        flags);
        PS_LAUNCH_CHECK();
    }
}

void launch_svd(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out, int dtype,
                double *partials, cudaStream_t st) {
    PS_CHECK(p.svd != nullptr, PAULI_EINVAL, "apply: the SVD plan is missing (internal)");
    const SvdPlan &sp = *p.svd;
    PS_CHECK(out != nullptr || svd_batches(&sp) <= 1, PAULI_EUNSUPPORTED,
             "apply: the SVD gather of this operator runs in several batches and needs an output vector");
#define PS_S(T)                                                                      \
    do {                                                                             \
        if (dtype == PAULI_C64) launch_svd_t<float, T>(cfg, sp, v, in, out, partials, st); \
        else launch_svd_t<double, T>(cfg, sp, v, in, out, partials, st);                  \
    } while (0)
    if (cfg.tpt == 4) PS_S(4);
    else if (cfg.tpt == 2) PS_S(2);
    else PS_S(1);
#undef PS_S
}

}  // namespace ps
