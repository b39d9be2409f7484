// build.cu -- Pauli-sum construction on the GPU:
//   * symplectic-form conversion of input terms (Sec. 2.2.2),
//   * Jordan-Wigner raw entries straight from bitwise products
//     (Algorithm 1 with eq. pauli_prod_x / pauli_prod_z / pauli_prod_phase),
//   * canonical reduction: stable radix sort on (X, Z), in-order duplicate
//     sums, drop below eps (Sec. 2.3),
//   * X-mask groups (eq. topological_group) and the per-split apply plan.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ps_internal.cuh"

namespace ps {
namespace {

__device__ __forceinline__ double2 ipow_mul(double2 c, int k) {
    switch (k & 3) {
        case 0: return c;
        case 1: return make_double2(-c.y, c.x);
        case 2: return make_double2(-c.x, -c.y);
        default: return make_double2(c.y, -c.x);
    }
}

// C = i^gamma * c * (letter ? i^popcount(x & z) : 1)
__global__ void k_to_xz(int64_t m, const uint64_t *x, const uint64_t *z, const uint8_t *gamma,
                        const double *cre, const double *cim, int letter, double2 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int k = gamma ? (int)gamma[i] : 0;
    if (letter) k += __popcll(x[i] & z[i]);
    out[i] = ipow_mul(make_double2(cre[i], cim[i]), k);
}

// ---------------------------------------------------------------------------
// Jordan-Wigner.  In XZ form a ladder operator is
//   a_P^dagger = 1/2 X^{e_P} Z^{below} + 1/2 X^{e_P} Z^{below | e_P}
//   a_P        = 1/2 X^{e_P} Z^{below} - 1/2 X^{e_P} Z^{below | e_P}
// (the Y letter -/+ i/2 Y_P carries i^#Y = i into XZ form).  A product of
// factors multiplies left to right with
//   (X^a Z^b)(X^c Z^d) = (-1)^popcount(b & c) X^(a^c) Z^(b^d).
// ---------------------------------------------------------------------------
struct Factor {
    int P;
    int dag;
};

__device__ __forceinline__ int64_t expand(const Factor *f, int nf, double2 scale, int64_t pos,
                                          uint64_t *ox, uint64_t *oz, double2 *oc) {
    const int ne = 1 << nf;
    for (int e = 0; e < ne; ++e) {
        uint64_t x = 0, z = 0;
        int neg = 0;
        double mag = 1.0;
        for (int j = 0; j < nf; ++j) {
            const int sel = (e >> (nf - 1 - j)) & 1;
            const uint64_t bit = 1ull << f[j].P;
            const uint64_t fx = bit;
            const uint64_t fz = (bit - 1ull) | (sel ? bit : 0ull);
            neg ^= __popcll(z & fx) & 1;  // eq. pauli_prod_phase
            x ^= fx;
            z ^= fz;
            if (sel && !f[j].dag) neg ^= 1;  // -1/2 for the Z-carrying term of a_P
            mag *= 0.5;
        }
        const double s = neg ? -mag : mag;
        ox[pos] = x;
        oz[pos] = z;
        oc[pos] = make_double2(scale.x * s, scale.y * s);
        ++pos;
    }
    return pos;
}

// slot layout: [e_nn] [one-body: (s*norb + p)*norb + q] [two-body: ((((s*2+t)*norb+p)*norb+q)*norb+r)*norb+u]
__global__ void k_jw_count(int norb, const double *h, const double *g, double e_nn, double eps,
                           int64_t nslots, int64_t *cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nslots) return;
    if (i == 0) {
        cnt[0] = (e_nn != 0.0) ? 1 : 0;
        return;
    }
    int64_t j = i - 1;
    const int64_t n1 = 2ll * norb * norb;
    if (j < n1) {
        int q = (int)(j % norb);
        int p = (int)((j / norb) % norb);
        cnt[i] = (fabs(h[p * norb + q]) > eps) ? 4 : 0;
        return;
    }
    j -= n1;
    int u = (int)(j % norb); j /= norb;
    int r = (int)(j % norb); j /= norb;
    int q = (int)(j % norb); j /= norb;
    int p = (int)(j % norb); j /= norb;
    int t = (int)(j % 2); j /= 2;
    int s = (int)j;
    int P = s * norb + p, Q = s * norb + q, R = t * norb + r, U = t * norb + u;
    double v = g[(((int64_t)p * norb + q) * norb + r) * norb + u];
    cnt[i] = (P != R && Q != U && fabs(v) > eps) ? 16 : 0;
}

__global__ void k_jw_expand(int norb, const double *h, const double *g, double e_nn,
                            int64_t nslots, const int64_t *cnt, const int64_t *off, uint64_t *ox,
                            uint64_t *oz, double2 *oc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nslots || cnt[i] == 0) return;
    int64_t pos = off[i];
    if (i == 0) {
        ox[pos] = 0;
        oz[pos] = 0;
        oc[pos] = make_double2(e_nn, 0.0);
        return;
    }
    int64_t j = i - 1;
    const int64_t n1 = 2ll * norb * norb;
    Factor f[4];
    if (j < n1) {
        int q = (int)(j % norb);
        int p = (int)((j / norb) % norb);
        int s = (int)(j / ((int64_t)norb * norb));
        f[0] = {s * norb + p, 1};
        f[1] = {s * norb + q, 0};
        expand(f, 2, make_double2(h[p * norb + q], 0.0), pos, ox, oz, oc);
        return;
    }
    j -= n1;
    int u = (int)(j % norb); j /= norb;
    int r = (int)(j % norb); j /= norb;
    int q = (int)(j % norb); j /= norb;
    int p = (int)(j % norb); j /= norb;
    int t = (int)(j % 2); j /= 2;
    int s = (int)j;
    double v = g[(((int64_t)p * norb + q) * norb + r) * norb + u];
    f[0] = {s * norb + p, 1};
    f[1] = {t * norb + r, 1};
    f[2] = {t * norb + u, 0};
    f[3] = {s * norb + q, 0};
    expand(f, 4, make_double2(0.5 * v, 0.0), pos, ox, oz, oc);
}

__global__ void k_fermion_expand(int nterms, const int *nf, const int *fstart, const int *modes,
                                 const int *dag, const double *cre, const double *cim,
                                 const int64_t *off, uint64_t *ox, uint64_t *oz, double2 *oc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nterms) return;
    Factor f[8];
    for (int j = 0; j < nf[t]; ++j) f[j] = {modes[fstart[t] + j], dag[fstart[t] + j]};
    expand(f, nf[t], make_double2(cre[t], cim[t]), off[t], ox, oz, oc);
}

// ---------------------------------------------------------------------------
// canonical reduction
// ---------------------------------------------------------------------------
__global__ void k_head_flags(const uint64_t *a, const uint64_t *b, int64_t n, int64_t *flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || a[i] != a[i - 1] || (b && b[i] != b[i - 1])) ? 1 : 0;
}

__global__ void k_run_starts(const int64_t *flag, const int64_t *id, int64_t n, int64_t *start) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) start[id[i]] = i;
}

// one thread per run: left-to-right sum in stable (input) order, then the drop test
__global__ void k_run_sums(int64_t nruns, int64_t n, const int64_t *start, const int64_t *perm,
                           const double2 *c, double eps2, double2 *sum, int64_t *keep) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    int64_t a = start[r], b = (r + 1 < nruns) ? start[r + 1] : n;
    double2 s = c[perm[a]];
    for (int64_t j = a + 1; j < b; ++j) {
        double2 v = c[perm[j]];
        s.x = __dadd_rn(s.x, v.x);
        s.y = __dadd_rn(s.y, v.y);
    }
    sum[r] = s;
    double mag2 = __dadd_rn(__dmul_rn(s.x, s.x), __dmul_rn(s.y, s.y));
    keep[r] = (mag2 > eps2) ? 1 : 0;
}

__global__ void k_compact(int64_t nruns, const int64_t *start, const int64_t *keep,
                          const int64_t *pos, const uint64_t *kx, const uint64_t *kz,
                          const double2 *sum, uint64_t *ox, uint64_t *oz, double2 *oc) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns || !keep[r]) return;
    int64_t o = pos[r];
    ox[o] = kx[start[r]];
    oz[o] = kz[start[r]];
    oc[o] = sum[r];
}

// properties of the reduced sum: any imaginary part, the largest |C|, and the
// largest imaginary part of a letter-form coefficient c = C i^-popcount(x&z)
__global__ void k_props(int64_t m, const uint64_t *x, const uint64_t *z, const double2 *c,
                        unsigned long long *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 v = c[i];
    if (v.y != 0.0) atomicOr(&out[0], 1ull);
    double mag = sqrt(v.x * v.x + v.y * v.y);
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(mag));
    int k = __popcll(x[i] & z[i]) & 1;
    double im_letter = fabs(k ? v.x : v.y);
    atomicMax(&out[2], (unsigned long long)__double_as_longlong(im_letter));
}

// ---------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------
__global__ void k_fill_group_id(int64_t G, const int64_t *gstart, int64_t *gid) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    for (int64_t t = gstart[g]; t < gstart[g + 1]; ++t) gid[t] = g;
}

// Low Z mask of a term in a merged plan.  When a target t and its source
// s = t ^ x have the same low-half popcount (both in one block of a
// single-block sector), exactly half of the bits of x_lo are set in s, so
// (-1)^popc((z ^ x_lo) & s) = (-1)^(popc(x_lo) / 2) (-1)^popc(z & s) on every
// pair the sector keeps: the masks z_lo and z_lo ^ x_lo merge into one segment
// (the smaller of the two) with that sign on the other's coefficients.  For an
// odd popc(x_lo) no pair stays in the block; its terms are left as they are.
__device__ __forceinline__ uint64_t merged_zlo(uint64_t zlo, uint64_t xlo, bool merge, bool &neg) {
    neg = false;
    if (!merge || (__popcll(xlo) & 1)) return zlo;
    const uint64_t alt = zlo ^ xlo;
    if (alt < zlo) {
        neg = (__popcll(xlo) >> 1) & 1;
        return alt;
    }
    return zlo;
}

// sort key of a term inside the plan: (group id, z_lo, z_hi)
__global__ void k_plan_keys(int64_t m, int n_lo, int n_hi, const int64_t *gid, const uint64_t *x, const uint64_t *z,
                            int merge, uint64_t *khi, uint64_t *klo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t lomask = (n_lo >= 64) ? ~0ull : ((1ull << n_lo) - 1ull);
    bool neg;
    uint64_t zlo = merged_zlo(z[i] & lomask, x[i] & lomask, merge != 0, neg);
    uint64_t zhi = z[i] >> n_lo;
    khi[i] = (uint64_t)gid[i];
    klo[i] = (zlo << n_hi) | zhi;
}

__global__ void k_plan_terms(int64_t m, int n_lo, int n_hi, const uint64_t *klo, const int64_t *perm,
                             const uint64_t *x, const uint64_t *z, int merge, const double2 *c, uint32_t *t_zhi,
                             double2 *t_c64, float2 *t_c32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t hmask = (n_hi >= 64) ? ~0ull : ((1ull << n_hi) - 1ull);
    uint64_t lomask = (n_lo >= 64) ? ~0ull : ((1ull << n_lo) - 1ull);
    t_zhi[i] = (uint32_t)(klo[i] & hmask);
    const int64_t o = perm[i];
    double2 v = c[o];
    bool neg;
    (void)merged_zlo(z[o] & lomask, x[o] & lomask, merge != 0, neg);
    if (neg) {
        v.x = -v.x;
        v.y = -v.y;
    }
    t_c64[i] = v;
    t_c32[i] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_plan_segments(int64_t m, int n_hi, const int64_t *head, const int64_t *sid,
                                const uint64_t *khi, const uint64_t *klo, int32_t *s_t0,
                                uint32_t *s_zlo, int64_t *seg_group) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m || !head[i]) return;
    int64_t s = sid[i];
    s_t0[s] = (int32_t)i;
    s_zlo[s] = (uint32_t)(klo[i] >> n_hi);
    seg_group[s] = (int64_t)khi[i];
}

__global__ void k_plan_group_segs(int64_t S, const int64_t *seg_group, int32_t *g_s0) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (s == 0 || seg_group[s] != seg_group[s - 1]) g_s0[seg_group[s]] = (int32_t)s;
}

__global__ void k_shift_right(int64_t m, const uint64_t *in, int sh, uint64_t *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = (sh >= 64) ? 0ull : (in[i] >> sh);
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <typename T>
T *alloc_copy_d2d(const Allocator &al, const T *src, int64_t n, cudaStream_t st) {
    T *p = static_cast<T *>(dev_alloc(al, (n > 0 ? n : 1) * sizeof(T)));
    if (n > 0) PS_CUDA(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    return p;
}

}  // namespace

// ---------------------------------------------------------------------------
void canonicalize(pauli_sum *h, int64_t m, uint64_t *d_x, uint64_t *d_z, double2 *d_c,
                  double eps_drop, cudaStream_t st) {
    const Allocator &al = h->al;
    h->m = 0;
    h->G = 0;
    if (m > 0) {
        DevBuf<uint64_t> kx(al, m), kz(al, m);
        DevBuf<int64_t> perm(al, m), flag(al, m), id(al, m);
        PS_CUDA(cudaMemcpyAsync(kx.p, d_x, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        PS_CUDA(cudaMemcpyAsync(kz.p, d_z, m * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        radix_sort_keys(kx.p, kz.p, perm.p, m, h->n, h->n, al, st);
        k_head_flags<<<nblk(m), 256, 0, st>>>(kx.p, kz.p, m, flag.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(flag.p, id.p, m, al, st);
        int64_t last_id = 0, last_flag = 0;
        PS_CUDA(cudaMemcpyAsync(&last_id, id.p + m - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(&last_flag, flag.p + m - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        const int64_t nruns = last_id + last_flag;
        DevBuf<int64_t> start(al, nruns), keep(al, nruns), pos(al, nruns);
        DevBuf<double2> sum(al, nruns);
        k_run_starts<<<nblk(m), 256, 0, st>>>(flag.p, id.p, m, start.p);
        PS_LAUNCH_CHECK();
        k_run_sums<<<nblk(nruns), 256, 0, st>>>(nruns, m, start.p, perm.p, d_c, eps_drop * eps_drop,
                                               sum.p, keep.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(keep.p, pos.p, nruns, al, st);
        int64_t lp = 0, lk = 0;
        PS_CUDA(cudaMemcpyAsync(&lp, pos.p + nruns - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(&lk, keep.p + nruns - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        const int64_t M = lp + lk;
        h->m = M;
        h->x = static_cast<uint64_t *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(uint64_t)));
        h->z = static_cast<uint64_t *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(uint64_t)));
        h->c = static_cast<double2 *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(double2)));
        k_compact<<<nblk(nruns), 256, 0, st>>>(nruns, start.p, keep.p, pos.p, kx.p, kz.p, sum.p,
                                              h->x, h->z, h->c);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaStreamSynchronize(st));
    }
    if (!h->x) {
        h->x = static_cast<uint64_t *>(dev_alloc(al, sizeof(uint64_t)));
        h->z = static_cast<uint64_t *>(dev_alloc(al, sizeof(uint64_t)));
        h->c = static_cast<double2 *>(dev_alloc(al, sizeof(double2)));
    }
    // X-mask groups
    const int64_t M = h->m;
    if (M > 0) {
        DevBuf<int64_t> flag(al, M), id(al, M);
        k_head_flags<<<nblk(M), 256, 0, st>>>(h->x, nullptr, M, flag.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(flag.p, id.p, M, al, st);
        int64_t li = 0, lf = 0;
        PS_CUDA(cudaMemcpyAsync(&li, id.p + M - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(&lf, flag.p + M - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        const int64_t G = li + lf;
        h->G = G;
        h->gstart = static_cast<int64_t *>(dev_alloc(al, (G + 1) * sizeof(int64_t)));
        h->gx = static_cast<uint64_t *>(dev_alloc(al, G * sizeof(uint64_t)));
        k_run_starts<<<nblk(M), 256, 0, st>>>(flag.p, id.p, M, h->gstart);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaMemcpyAsync(h->gstart + G, &M, sizeof(int64_t), cudaMemcpyHostToDevice, st));
        // group x = x of its first term
        std::vector<int64_t> gs(G + 1);
        PS_CUDA(cudaMemcpyAsync(gs.data(), h->gstart, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        std::vector<uint64_t> hx(M);
        PS_CUDA(cudaMemcpy(hx.data(), h->x, M * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        std::vector<uint64_t> gx(G);
        for (int64_t g = 0; g < G; ++g) gx[g] = hx[gs[g]];
        PS_CUDA(cudaMemcpy(h->gx, gx.data(), G * sizeof(uint64_t), cudaMemcpyHostToDevice));
        DevBuf<unsigned long long> props(al, 3);
        PS_CUDA(cudaMemsetAsync(props.p, 0, 3 * sizeof(unsigned long long), st));
        k_props<<<nblk(M), 256, 0, st>>>(M, h->x, h->z, h->c, props.p);
        PS_LAUNCH_CHECK();
        unsigned long long hp[3];
        PS_CUDA(cudaMemcpyAsync(hp, props.p, sizeof(hp), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        double cmax, imax;
        memcpy(&cmax, &hp[1], sizeof(double));
        memcpy(&imax, &hp[2], sizeof(double));
        h->real = (hp[0] == 0);
        h->cmax = cmax;
        h->hermitian = imax <= 1e-12 * cmax;
    } else {
        h->gstart = static_cast<int64_t *>(dev_alloc(al, sizeof(int64_t)));
        h->gx = static_cast<uint64_t *>(dev_alloc(al, sizeof(uint64_t)));
        PS_CUDA(cudaMemsetAsync(h->gstart, 0, sizeof(int64_t), st));
        h->real = true;
        h->hermitian = true;
        PS_CUDA(cudaStreamSynchronize(st));
    }
}

void to_xz_device(int64_t m, const uint64_t *x, const uint64_t *z, const uint8_t *gamma,
                  const double *cre, const double *cim, int letter, double2 *out, cudaStream_t st) {
    if (m <= 0) return;
    k_to_xz<<<nblk(m), 256, 0, st>>>(m, x, z, gamma, cre, cim, letter, out);
    PS_LAUNCH_CHECK();
}

void jw_molecular_raw_device(int norb, const double *h, const double *g, double e_nn, double eps_int,
                             const Allocator &al, DevBuf<uint64_t> &x, DevBuf<uint64_t> &z,
                             DevBuf<double2> &c, int64_t &count, cudaStream_t st) {
    const int64_t n1 = 2ll * norb * norb;
    const int64_t n4 = (int64_t)norb * norb * norb * norb;
    const int64_t nslots = 1 + n1 + 4 * n4;
    DevBuf<double> dh(al, (size_t)norb * norb), dg(al, (size_t)n4);
    PS_CUDA(cudaMemcpyAsync(dh.p, h, norb * norb * sizeof(double), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(dg.p, g, n4 * sizeof(double), cudaMemcpyHostToDevice, st));
    DevBuf<int64_t> cnt(al, nslots), off(al, nslots);
    k_jw_count<<<nblk(nslots), 256, 0, st>>>(norb, dh.p, dg.p, e_nn, eps_int, nslots, cnt.p);
    PS_LAUNCH_CHECK();
    exclusive_scan_i64(cnt.p, off.p, nslots, al, st);
    int64_t lo = 0, lc = 0;
    PS_CUDA(cudaMemcpyAsync(&lo, off.p + nslots - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaMemcpyAsync(&lc, cnt.p + nslots - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PS_CUDA(cudaStreamSynchronize(st));
    count = lo + lc;
    x = DevBuf<uint64_t>(al, count);
    z = DevBuf<uint64_t>(al, count);
    c = DevBuf<double2>(al, count);
    k_jw_expand<<<nblk(nslots), 256, 0, st>>>(norb, dh.p, dg.p, e_nn, nslots, cnt.p, off.p, x.p, z.p,
                                              c.p);
    PS_LAUNCH_CHECK();
    PS_CUDA(cudaStreamSynchronize(st));
}

void jw_fermion_raw_device(int n, int nterms, const int *nf, const int *modes, const int *dag,
                           const double *cre, const double *cim, const Allocator &al,
                           DevBuf<uint64_t> &x, DevBuf<uint64_t> &z, DevBuf<double2> &c,
                           int64_t &count, cudaStream_t st) {
    (void)n;
    std::vector<int> fstart(nterms + 1, 0);
    std::vector<int64_t> off(nterms, 0);
    count = 0;
    for (int t = 0; t < nterms; ++t) {
        fstart[t + 1] = fstart[t] + nf[t];
        off[t] = count;
        count += (int64_t)1 << nf[t];
    }
    const int nfac = fstart[nterms];
    DevBuf<int> d_nf(al, nterms), d_fs(al, nterms + 1), d_modes(al, nfac), d_dag(al, nfac);
    DevBuf<double> d_re(al, nterms), d_im(al, nterms);
    DevBuf<int64_t> d_off(al, nterms);
    PS_CUDA(cudaMemcpyAsync(d_nf.p, nf, nterms * sizeof(int), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(d_fs.p, fstart.data(), (nterms + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    if (nfac > 0) {
        PS_CUDA(cudaMemcpyAsync(d_modes.p, modes, nfac * sizeof(int), cudaMemcpyHostToDevice, st));
        PS_CUDA(cudaMemcpyAsync(d_dag.p, dag, nfac * sizeof(int), cudaMemcpyHostToDevice, st));
    }
    PS_CUDA(cudaMemcpyAsync(d_re.p, cre, nterms * sizeof(double), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(d_im.p, cim, nterms * sizeof(double), cudaMemcpyHostToDevice, st));
    PS_CUDA(cudaMemcpyAsync(d_off.p, off.data(), nterms * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    x = DevBuf<uint64_t>(al, count);
    z = DevBuf<uint64_t>(al, count);
    c = DevBuf<double2>(al, count);
    k_fermion_expand<<<nblk(nterms), 256, 0, st>>>(nterms, d_nf.p, d_fs.p, d_modes.p, d_dag.p, d_re.p,
                                                   d_im.p, d_off.p, x.p, z.p, c.p);
    PS_LAUNCH_CHECK();
    PS_CUDA(cudaStreamSynchronize(st));
}

// T(t_lo) over the x = 0 group's terms with z_hi = 0 (the first term of a
// segment, terms being sorted by z_hi inside it), FP64 sums in segment order
__global__ void k_diag_table(int n_lo, int nseg, const int32_t *s_t0, const uint32_t *s_zlo,
                             const uint32_t *t_zhi, const double2 *t_c64, double2 *tab64, float2 *tab32) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = 1u << n_lo;
    if (t >= n) return;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < nseg; ++s) {
        const int t0 = s_t0[s];
        if (t_zhi[t0] != 0u) continue;
        const double2 c = t_c64[t0];
        const bool neg = __popc(s_zlo[s] & t) & 1;
        re += neg ? -c.x : c.x;
        im += neg ? -c.y : c.y;
    }
    tab64[t] = make_double2(re, im);
    const float hr = (float)re, hi = (float)im;
    tab32[t] = make_float2(hr, hi);
    tab32[n + t] = make_float2((float)(re - (double)hr), (float)(im - (double)hi));
}

void free_plan(const Allocator &al, Plan &p) {
    dev_free(al, p.pc_xhi); dev_free(al, p.pc_i0); dev_free(al, p.it_xlo); dev_free(al, p.it_s0);
    dev_free(al, p.pc_lofree);
    dev_free(al, p.it_xhi);
    dev_free(al, p.s_xhi);
    dev_free(al, p.s_zlo); dev_free(al, p.s_t0);
    dev_free(al, p.t_zhi); dev_free(al, p.t_c64); dev_free(al, p.t_c32);
    dev_free(al, p.diag_tab64); dev_free(al, p.diag_tab32); dev_free(al, p.diag_rest);
    free_local_plan(p.local);
    free_local_plan(p.local_cl);
    free_lists(al, p);
    dev_free(al, p.partials);
    dev_free(al, p.split_buf);
    dev_free(al, p.df_buf);
    free_svd_plan(p.svd);
    p = Plan();
}

Plan *find_plan(pauli_sum *h, const SectorView &v) {
    const bool merged = plan_merges(v);
    for (int i = 0; i < h->nplans; ++i)
        if (h->plans[i].n_lo == v.n_lo && h->plans[i].merged == merged) return &h->plans[i];
    return nullptr;
}

Plan &get_plan(pauli_sum *h, const SectorView &v, cudaStream_t st) {
    const int n_lo = v.n_lo;
    const bool merged = plan_merges(v);
    for (int i = 0; i < h->nplans; ++i)
        if (h->plans[i].n_lo == n_lo && h->plans[i].merged == merged) return h->plans[i];
    if (h->nplans == 4) {  // evict the oldest
        free_plan(h->al, h->plans[0]);
        for (int i = 1; i < 4; ++i) h->plans[i - 1] = h->plans[i];
        h->plans[3] = Plan();
        h->nplans = 3;
    }
    const Allocator &al = h->al;
    const int n_hi = h->n - n_lo;
    const int64_t M = h->m, G = h->G;
    Plan p;
    p.n_lo = n_lo;
    p.merged = merged;
    p.M = M;
    p.G = G;
    p.real = h->real;
    p.t_zhi = static_cast<uint32_t *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(uint32_t)));
    p.t_c64 = static_cast<double2 *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(double2)));
    p.t_c32 = static_cast<float2 *>(dev_alloc(al, (M > 0 ? M : 1) * sizeof(float2)));
    std::vector<int32_t> g_s0(G + 1, 0);
    int64_t S = 0;
    if (M > 0) {
        DevBuf<int64_t> gid(al, M), perm(al, M), head(al, M), sid(al, M);
        DevBuf<uint64_t> khi(al, M), klo(al, M), seg_key(al, M);
        k_fill_group_id<<<nblk(G), 256, 0, st>>>(G, h->gstart, gid.p);
        PS_LAUNCH_CHECK();
        k_plan_keys<<<nblk(M), 256, 0, st>>>(M, n_lo, n_hi, gid.p, h->x, h->z, merged ? 1 : 0, khi.p, klo.p);
        PS_LAUNCH_CHECK();
        int gbits = 1;
        while ((1ll << gbits) <= G) ++gbits;
        radix_sort_keys(khi.p, klo.p, perm.p, M, gbits, h->n, al, st);
        k_plan_terms<<<nblk(M), 256, 0, st>>>(M, n_lo, n_hi, klo.p, perm.p, h->x, h->z, merged ? 1 : 0, h->c,
                                              p.t_zhi, p.t_c64, p.t_c32);
        PS_LAUNCH_CHECK();
        // segments: runs of equal (group, z_lo) in the re-sorted order
        k_shift_right<<<nblk(M), 256, 0, st>>>(M, klo.p, n_hi, seg_key.p);
        PS_LAUNCH_CHECK();
        k_head_flags<<<nblk(M), 256, 0, st>>>(khi.p, seg_key.p, M, head.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(head.p, sid.p, M, al, st);
        int64_t ls = 0, lh = 0;
        PS_CUDA(cudaMemcpyAsync(&ls, sid.p + M - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaMemcpyAsync(&lh, head.p + M - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        S = ls + lh;
        p.s_zlo = static_cast<uint32_t *>(dev_alloc(al, S * sizeof(uint32_t)));
        p.s_t0 = static_cast<int32_t *>(dev_alloc(al, (S + 1) * sizeof(int32_t)));
        DevBuf<int64_t> seg_group(al, S);
        DevBuf<int32_t> d_gs0(al, G + 1);
        k_plan_segments<<<nblk(M), 256, 0, st>>>(M, n_hi, head.p, sid.p, khi.p, klo.p, p.s_t0, p.s_zlo,
                                                  seg_group.p);
        PS_LAUNCH_CHECK();
        int32_t m32 = (int32_t)M;
        PS_CUDA(cudaMemcpyAsync(p.s_t0 + S, &m32, sizeof(int32_t), cudaMemcpyHostToDevice, st));
        k_plan_group_segs<<<nblk(S), 256, 0, st>>>(S, seg_group.p, d_gs0.p);
        PS_LAUNCH_CHECK();
        PS_CUDA(cudaMemcpyAsync(g_s0.data(), d_gs0.p, G * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PS_CUDA(cudaStreamSynchronize(st));
        g_s0[G] = (int32_t)S;
    } else {
        p.s_zlo = static_cast<uint32_t *>(dev_alloc(al, sizeof(uint32_t)));
        p.s_t0 = static_cast<int32_t *>(dev_alloc(al, sizeof(int32_t)));
        PS_CUDA(cudaMemset(p.s_t0, 0, sizeof(int32_t)));
    }
    p.S = S;
    std::vector<uint64_t> gx(G > 0 ? G : 1);
    if (G > 0) PS_CUDA(cudaMemcpy(gx.data(), h->gx, G * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    const uint64_t lomask = (n_lo >= 64) ? ~0ull : ((1ull << n_lo) - 1ull);
    // pieces of consecutive groups with one x_hi; items of at most kSegsPerPiece segments
    std::vector<uint32_t> pc_xhi, it_xlo, it_xhi;
    std::vector<int32_t> pc_i0, it_s0;
    int items_in_piece = 0, segs_in_piece = 0;
    uint64_t cur_xhi = ~0ull;
    for (int64_t g = 0; g < G; ++g) {
        const uint64_t xhi = gx[g] >> n_lo, xlo = gx[g] & lomask;
        int32_t s = g_s0[g];
        const int32_t se = g_s0[g + 1];
        while (s < se) {
            const int32_t take = std::min<int32_t>(se - s, PlanLimits::kSegsPerPiece);
            if (pc_xhi.empty() || xhi != cur_xhi || items_in_piece == PlanLimits::kItemsPerPiece ||
                segs_in_piece + take > PlanLimits::kSegsPerPiece) {
                pc_xhi.push_back((uint32_t)xhi);
                pc_i0.push_back((int32_t)it_xlo.size());
                cur_xhi = xhi;
                items_in_piece = 0;
                segs_in_piece = 0;
            }
            it_xlo.push_back((uint32_t)xlo);
            it_xhi.push_back((uint32_t)xhi);
            it_s0.push_back(s);
            ++items_in_piece;
            segs_in_piece += take;
            s += take;
        }
    }
    pc_i0.push_back((int32_t)it_xlo.size());
    it_s0.push_back((int32_t)S);
    p.P = (int64_t)pc_xhi.size();
    p.I = (int64_t)it_xlo.size();
    // work estimate of a piece for one target: staging plus, per item, the gather
    // and one parity-add per segment
    p.h_pc_cumw.assign(p.P + 1, 0);
    for (int64_t q = 0; q < p.P; ++q) {
        int64_t wq = 8;
        for (int32_t it = pc_i0[q]; it < pc_i0[q + 1]; ++it) wq += 4 + (it_s0[it + 1] - it_s0[it]);
        p.h_pc_cumw[q + 1] = p.h_pc_cumw[q] + wq;
    }
    p.nseg_diag = (G > 0 && gx[0] == 0) ? g_s0[1] - g_s0[0] : 0;
    // pieces whose sources sit in the target's own columns (x_lo = 0 throughout),
    // without the x = 0 group (its segments keep the staged, compensated path)
    std::vector<uint8_t> pc_lofree(p.P > 0 ? p.P : 1, 0);
    for (int64_t q = 0; q < p.P; ++q) {
        bool lf = true;
        for (int32_t it = pc_i0[q]; it < pc_i0[q + 1] && lf; ++it)
            lf = it_xlo[it] == 0 && it_s0[it] >= p.nseg_diag;
        pc_lofree[q] = lf ? 1 : 0;
    }
    auto upload = [&](const void *src, size_t bytes) {
        void *d = dev_alloc(al, bytes > 0 ? bytes : 4);
        if (bytes > 0) PS_CUDA(cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
        return d;
    };
    p.pc_xhi = static_cast<uint32_t *>(upload(pc_xhi.data(), pc_xhi.size() * sizeof(uint32_t)));
    p.pc_i0 = static_cast<int32_t *>(upload(pc_i0.data(), pc_i0.size() * sizeof(int32_t)));
    p.pc_lofree = static_cast<uint8_t *>(upload(pc_lofree.data(), (size_t)p.P * sizeof(uint8_t)));
    p.it_xlo = static_cast<uint32_t *>(upload(it_xlo.data(), it_xlo.size() * sizeof(uint32_t)));
    p.it_xhi = static_cast<uint32_t *>(upload(it_xhi.data(), it_xhi.size() * sizeof(uint32_t)));
    {
        std::vector<uint32_t> s_xhi(S > 0 ? S : 1, 0);
        for (size_t it = 0; it < it_xhi.size(); ++it)
            for (int32_t s = it_s0[it]; s < it_s0[it + 1]; ++s) s_xhi[s] = it_xhi[it];
        p.s_xhi = static_cast<uint32_t *>(upload(s_xhi.data(), (S > 0 ? S : 0) * sizeof(uint32_t)));
    }
    p.it_s0 = static_cast<int32_t *>(upload(it_s0.data(), it_s0.size() * sizeof(int32_t)));
    p.h_it_xlo = it_xlo;
    p.h_it_s0 = it_s0;
    p.h_pc_i0 = pc_i0;
    if (p.nseg_diag > 0 && n_lo <= kDiagTabBits) {
        // diagonal table, and the diagonal segments left with a z_hi != 0 term
        const int nd = p.nseg_diag;
        std::vector<int32_t> st0(nd + 1);
        PS_CUDA(cudaMemcpy(st0.data(), p.s_t0, (nd + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        const int32_t nt = st0[nd] - st0[0];
        std::vector<uint32_t> tzhi(nt > 0 ? nt : 1);
        if (nt > 0) PS_CUDA(cudaMemcpy(tzhi.data(), p.t_zhi + st0[0], nt * sizeof(uint32_t), cudaMemcpyDeviceToHost));
        std::vector<int32_t> rest;
        for (int sg = 0; sg < nd; ++sg) {
            const int32_t a = st0[sg] - st0[0], b = st0[sg + 1] - st0[0];
            if (b - a >= 2 || (b - a == 1 && tzhi[a] != 0u)) rest.push_back(sg);
        }
        const int64_t ntab = 1ll << n_lo;
        p.diag_tab64 = static_cast<double2 *>(dev_alloc(al, ntab * sizeof(double2)));
        p.diag_tab32 = static_cast<float2 *>(dev_alloc(al, 2 * ntab * sizeof(float2)));
        k_diag_table<<<nblk(ntab), 256, 0, st>>>(n_lo, nd, p.s_t0, p.s_zlo, p.t_zhi, p.t_c64, p.diag_tab64,
                                                  p.diag_tab32);
        PS_CUDA(cudaGetLastError());
        p.n_diag_rest = (int32_t)rest.size();
        p.diag_rest = static_cast<int32_t *>(upload(rest.data(), rest.size() * sizeof(int32_t)));
        PS_CUDA(cudaStreamSynchronize(st));
    }
    h->plans[h->nplans] = p;
    return h->plans[h->nplans++];
}

}  // namespace ps
