// rows.cu -- the target-driven gather of eq. reverse_sum evaluated only at a
// list of target indices:
//
//   (H psi)_t = sum_g f_g(t XOR x_g) psi[t XOR x_g],
//   f_g(s)    = sum_{k in g} C_k (-1)^popcount(z_k & s),
//
// one CTA per listed target.  The CTA's threads take the groups in a fixed
// stride, the per-thread sums are combined by a fixed tree, so every result
// is reproducible.  A variational state that lives on a small set of
// configurations (the seniority-zero strings a pair-double ansatz reaches)
// needs H psi only there: <psi|H|psi> and the adjoint gradient's
// lam = P H psi come from these rows alone.
#include "apply_kernels.cuh"

namespace ps {
namespace {

constexpr int kRowThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kRowThreads)
k_apply_rows(SectorView v, int64_t G, const uint64_t *__restrict__ gx, const int64_t *__restrict__ gstart,
             const uint64_t *__restrict__ z, const double2 *__restrict__ c, const typename Cx<R>::T *__restrict__ psi,
             const int64_t *__restrict__ rows, typename Cx<R>::T *__restrict__ out, double *__restrict__ partials,
             int *status) {
    using C2 = typename Cx<R>::T;
    const int tid = threadIdx.x;
    const int64_t r = rows[blockIdx.x];
    if (r < 0 || r >= v.dim) {
        // an index outside the sector: nothing is read or written for it
        if (tid == 0) {
            atomicCAS(status, 0, (int)PAULI_EINVAL);
            if (partials) {
                double *q = partials + (int64_t)blockIdx.x * 4;
                q[0] = q[1] = q[2] = q[3] = 0.0;
            }
        }
        return;
    }
    // the target configuration t of sector index r
    uint64_t t;
    if (v.kind == PAULI_SECTOR_FULL) {
        t = (uint64_t)r;
    } else {
        int b = 0;
        while (b + 1 < v.nblk && v.off[b + 1] <= r) ++b;
        const int64_t rem = r - v.off[b];
        const int64_t rhi = rem / v.dlo[b], rlo = rem - rhi * v.dlo[b];
        const uint32_t thi = __ldg(v.list_hi + v.lst_hi_off[b] + rhi);
        const uint32_t tlo = __ldg(v.list_lo + v.lst_lo_off[b] + rlo);
        t = (uint64_t)tlo | ((uint64_t)thi << v.n_lo);
    }
    const uint64_t lomask = (1ull << v.n_lo) - 1ull;
    R ar = R(0), ai = R(0);
    for (int64_t g = tid; g < G; g += kRowThreads) {
        const uint64_t s = t ^ __ldg(gx + g);
        int64_t sidx;
        if (v.kind == PAULI_SECTOR_FULL) {
            sidx = (int64_t)s;
        } else {
            const uint32_t slo = (uint32_t)(s & lomask), shi = (uint32_t)(s >> v.n_lo);
            const int bb = v.blk_of_khi[cls_hi(v, shi)];
            if (bb < 0 || cls_lo(v, slo) != v.klo[bb]) continue;  // the source is outside the sector
            sidx = v.off[bb] + (int64_t)__ldg(v.rank_hi + shi) * v.dlo[bb] + (int64_t)__ldg(v.rank_lo + slo);
        }
        R fr = R(0), fi = R(0);
        const int64_t k1 = __ldg(gstart + g + 1);
        for (int64_t k = __ldg(gstart + g); k < k1; ++k) {
            const uint32_t par = __popcll(__ldg(z + k) & s);
            const double2 cc = __ldg(c + k);
            fr += flip((R)cc.x, par);
            fi += flip((R)cc.y, par);
        }
        const C2 a = psi[sidx];
        ar += fr * a.x - fi * a.y;
        ai += fr * a.y + fi * a.x;
    }
    // fixed-order combination: warp tree, then the warps in order (FP64)
    double hr = (double)ar, hi = (double)ai;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hr += __shfl_down_sync(0xffffffffu, hr, o);
        hi += __shfl_down_sync(0xffffffffu, hi, o);
    }
    __shared__ double red[2][kRowThreads / 32];
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red[0][warp] = hr;
        red[1][warp] = hi;
    }
    __syncthreads();
    if (tid == 0) {
        double sr = 0.0, si = 0.0;
        for (int w = 0; w < kRowThreads / 32; ++w) {
            sr += red[0][w];
            si += red[1][w];
        }
        C2 h;
        h.x = (R)sr;
        h.y = (R)si;
        if (out) out[r] = h;
        if (partials) {
            // the stored value's own rounding enters the sums (as for the full apply)
            const C2 p = psi[r];
            const double pr = (double)p.x, pi = (double)p.y, qr = (double)h.x, qi = (double)h.y;
            double *q = partials + (int64_t)blockIdx.x * 4;
            q[0] = pr * qr + pi * qi;   // Re conj(psi_t) (H psi)_t
            q[1] = pr * qi - pi * qr;   // Im
            q[2] = qr * qr + qi * qi;
            q[3] = pr * pr + pi * pi;
        }
    }
}

}  // namespace

void launch_apply_rows(const pauli_sum *H, const SectorView &v, const void *psi, const int64_t *rows, int64_t nrows,
                       void *out, int dtype, double *partials, cudaStream_t st) {
    PS_CHECK(nrows < (1ll << 31), PAULI_EUNSUPPORTED, "rows: at most 2^31 - 1 targets per call");
    if (nrows <= 0) return;
    const unsigned grid = (unsigned)nrows;
    if (dtype == PAULI_C64) {
        k_apply_rows<float><<<grid, kRowThreads, 0, st>>>(v, H->G, H->gx, H->gstart, H->z, H->c,
                                                          static_cast<const float2 *>(psi), rows,
                                                          static_cast<float2 *>(out), partials,
                                                          H->status);
    } else {
        k_apply_rows<double><<<grid, kRowThreads, 0, st>>>(v, H->G, H->gx, H->gstart, H->z, H->c,
                                                           static_cast<const double2 *>(psi), rows,
                                                           static_cast<double2 *>(out), partials,
                                                           H->status);
    }
    PS_LAUNCH_CHECK();
}

}  // namespace ps
