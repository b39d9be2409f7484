// krylov.cu -- real-time propagation psi <- exp(-i dt H) psi by an m-vector
// Lanczos (Krylov) projection, every scalar kept on the device so that a step
// can be captured once in a CUDA graph and replayed.
//
// The paper names Krylov-based solvers as users of the same operator engine
// (Sec. 4); the propagator follows the standard Lanczos construction:
//   v_0 = psi / beta_0,                         beta_0 = ||psi||
//   w_j = H v_j,  alpha_j = <v_j|w_j>,
//   w_j <- w_j - alpha_j v_j - beta_j v_{j-1},  beta_{j+1} = ||w_j||,
//   v_{j+1} = w_j / beta_{j+1},
//   psi(t+dt) = beta_0 V_m exp(-i dt T_m) e_0,  T_m = tridiag(beta, alpha, beta),
// with alpha_j from the FP64 reduction of the apply kernel (pauli_expect's
// epilogue), FP64 norms, and exp(-i dt T_m) e_0 from a cyclic Jacobi
// eigen-decomposition of the small real symmetric T_m on the device.  The
// vectors are stored unnormalised, u_j = beta_j v_j (j > 0): their scales enter
// the next update's coefficients and the final combination, so no pass over the
// state rescales them.
#include <cmath>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {
namespace {

constexpr int kVecThreads = 256;
constexpr int kMaxKrylov = 32;

// Device scalars of one Lanczos step.
struct KrylovScalars {
    double alpha[kMaxKrylov];
    double beta[kMaxKrylov + 1];   // beta[0] = ||psi||, beta[j+1] = ||w_j||
    double cre[kMaxKrylov], cim[kMaxKrylov];  // beta_0 exp(-i dt T) e_0
    double red[4];                 // output slot of the 4-wide reduction
};

template <typename R>
__device__ __forceinline__ void block_sum_store(double v, double *partials) {
    __shared__ double red[kVecThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kVecThreads / 32; ++w) s += red[w];
        partials[(int64_t)blockIdx.x * 4 + 0] = s;
        partials[(int64_t)blockIdx.x * 4 + 1] = 0.0;
        partials[(int64_t)blockIdx.x * 4 + 2] = 0.0;
        partials[(int64_t)blockIdx.x * 4 + 3] = 0.0;
    }
}

// Per-thread sum of |x_i|^2.  FP64 vectors: FP64.  FP32 vectors: each square
// split exactly into FP32 hi + lo (FMA) and added with TwoSum (compensated
// summation, error ~ one FP32 rounding of the thread's total), converted to
// FP64 for the block and grid reduction; FP64 arithmetic is slow on this GPU.
template <typename R> struct NormAcc;
template <> struct NormAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double2 v) { s += v.x * v.x + v.y * v.y; }
    __device__ __forceinline__ double get() const { return s; }
};
template <> struct NormAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void sq(float a) {
        const float p = __fmul_rn(a, a);
        const float e = __fmaf_rn(a, a, -p);
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float2 v) {
        sq(v.x);
        sq(v.y);
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// partial sums of ||x||^2
template <typename R>
__global__ void __launch_bounds__(kVecThreads) k_norm2(const typename Cx<R>::T *__restrict__ x, int64_t n,
                                                       double *partials) {
    NormAcc<R> acc;
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads)
        acc.add(x[i]);
    block_sum_store<R>(acc.get(), partials);
}

// y = x / sqrt(sc->red[0]) (zero if the norm vanished); records the norm in *beta_out
template <typename R>
__global__ void __launch_bounds__(kVecThreads) k_normalize(const typename Cx<R>::T *__restrict__ x,
                                                           typename Cx<R>::T *__restrict__ y, int64_t n,
                                                           KrylovScalars *sc, int beta_slot) {
    const double nrm = sqrt(sc->red[0]);
    const double inv = nrm > 1e-300 ? 1.0 / nrm : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->beta[beta_slot] = nrm;
    const R f = (R)inv;
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
        typename Cx<R>::T v = x[i];
        v.x *= f;
        v.y *= f;
        y[i] = v;
    }
}

// 1 / beta_j, the scale of the stored Lanczos vector u_j (v_j = u_j / beta_j;
// u_0 = v_0 is stored normalised)
__device__ __forceinline__ double lanczos_scale(const KrylovScalars *sc, int j) {
    if (j == 0) return 1.0;
    const double b = sc->beta[j];
    return b > 1e-300 ? 1.0 / b : 0.0;
}

// The Lanczos vectors are stored unnormalised (u_j = beta_j v_j for j > 0), which
// saves the pass that would rescale each of them.  On entry w = H u_j; on exit
//   w <- s_j (w - alpha_j u_j) - beta_j s_{j-1} u_{j-1} = H v_j - alpha_j v_j - beta_j v_{j-1}
// (= u_{j+1}), with s_j = 1 / beta_j and alpha_j = s_j^2 Re <u_j|H u_j> from the
// apply's FP64 expectation reduction left in sc->red; partial sums of ||w||^2.
template <typename R>
__global__ void __launch_bounds__(kVecThreads)
k_lanczos_update(typename Cx<R>::T *__restrict__ w, const typename Cx<R>::T *__restrict__ vj,
                 const typename Cx<R>::T *__restrict__ vjm1, int64_t n, KrylovScalars *sc, int j,
                 double *partials) {
    const double sj = lanczos_scale(sc, j);
    const double alpha = sc->red[0] * sj * sj;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->alpha[j] = alpha;
    const R c1 = (R)sj, c2 = (R)(alpha * sj);
    const R c3 = vjm1 ? (R)(sc->beta[j] * lanczos_scale(sc, j - 1)) : R(0);
    NormAcc<R> acc;
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
        typename Cx<R>::T x = w[i];
        const typename Cx<R>::T v = vj[i];
        x.x = c1 * x.x - c2 * v.x;
        x.y = c1 * x.y - c2 * v.y;
        if (vjm1) {
            const typename Cx<R>::T u = vjm1[i];
            x.x -= c3 * u.x;
            x.y -= c3 * u.y;
        }
        w[i] = x;
        acc.add(x);
    }
    block_sum_store<R>(acc.get(), partials);
}

// One CTA: eigen-decomposition of T_m by cyclic Jacobi rotations (FP64), then
// c = beta_0 Q exp(-i dt Lambda) Q^T e_0.  Thread 0 does the arithmetic (m <= 32).
__global__ void k_tridiag_expm(KrylovScalars *sc, int m, double dt) {
    if (threadIdx.x != 0) return;
    double A[kMaxKrylov][kMaxKrylov], Q[kMaxKrylov][kMaxKrylov];
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < m; ++k) {
            A[i][k] = 0.0;
            Q[i][k] = (i == k) ? 1.0 : 0.0;
        }
    for (int i = 0; i < m; ++i) A[i][i] = sc->alpha[i];
    for (int i = 0; i + 1 < m; ++i) A[i][i + 1] = A[i + 1][i] = sc->beta[i + 1];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < m; ++p) {
            diag += A[p][p] * A[p][p];
            for (int q = p + 1; q < m; ++q) off += A[p][q] * A[p][q];
        }
        if (off <= 1e-34 * (diag + 1e-300)) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p][q];
                if (fabs(apq) < 1e-300) continue;
                // rotation zeroing A[p][q]: tan(phi) = t, the smaller root of t^2 + 2 tau t - 1 = 0
                const double tau = (A[q][q] - A[p][p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < m; ++k) {  // A <- A J (columns p, q)
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {  // Q <- Q J
                    const double qkp = Q[k][p], qkq = Q[k][q];
                    Q[k][p] = c * qkp - s * qkq;
                    Q[k][q] = s * qkp + c * qkq;
                }
            }
    }
    const double b0 = sc->beta[0];
    for (int j = 0; j < m; ++j) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < m; ++k) {
            double sn, cs;
            sincos(-dt * A[k][k], &sn, &cs);
            const double wgt = Q[j][k] * Q[0][k];
            re += wgt * cs;
            im += wgt * sn;
        }
        sc->cre[j] = b0 * re;
        sc->cim[j] = b0 * im;
    }
}

// psi = sum_j c_j v_j.  FP64 vectors: FP64.  FP32 vectors: each c_j split
// once per block into FP32 hi + lo parts; per element the products are split
// exactly (FMA) and summed with TwoSum compensation, so the sum is about
// FP64-accurate before its final rounding to FP32.
template <typename R> struct CombineAcc;
template <> struct CombineAcc<double> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(const float4 &, double cr, double ci, double2 v) {
        re += cr * v.x - ci * v.y;
        im += cr * v.y + ci * v.x;
    }
    __device__ __forceinline__ double2 get() const { return make_double2(re, im); }
};
template <> struct CombineAcc<float> {
    float sr = 0.f, er = 0.f, si = 0.f, ei = 0.f;
    __device__ __forceinline__ static void acc(float &s, float &c, float p) {
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c = __fadd_rn(c, err);
    }
    // c4 = {Re c hi, Re c lo, Im c hi, Im c lo}
    __device__ __forceinline__ void add(const float4 &c4, double, double, float2 v) {
        const float p1 = __fmul_rn(c4.x, v.x), q1 = __fmaf_rn(c4.x, v.x, -p1);
        const float p2 = __fmul_rn(c4.z, v.y), q2 = __fmaf_rn(c4.z, v.y, -p2);
        const float p3 = __fmul_rn(c4.x, v.y), q3 = __fmaf_rn(c4.x, v.y, -p3);
        const float p4 = __fmul_rn(c4.z, v.x), q4 = __fmaf_rn(c4.z, v.x, -p4);
        acc(sr, er, p1);
        acc(sr, er, -p2);
        er = __fadd_rn(er, (q1 - q2) + (c4.y * v.x - c4.w * v.y));
        acc(si, ei, p3);
        acc(si, ei, p4);
        ei = __fadd_rn(ei, (q3 + q4) + (c4.y * v.y + c4.w * v.x));
    }
    __device__ __forceinline__ float2 get() const { return make_float2(sr + er, si + ei); }
};

template <typename R>
__global__ void __launch_bounds__(kVecThreads) k_krylov_combine(const typename Cx<R>::T *__restrict__ V, int64_t n,
                                                                int m, const KrylovScalars *sc,
                                                                typename Cx<R>::T *__restrict__ psi) {
    __shared__ double cr[kMaxKrylov], ci[kMaxKrylov];
    __shared__ float4 c4[kMaxKrylov];
    if (threadIdx.x < m) {
        // psi = sum_j c_j v_j = sum_j (c_j s_j) u_j
        const double sj = lanczos_scale(sc, threadIdx.x);
        const double a = sc->cre[threadIdx.x] * sj, b = sc->cim[threadIdx.x] * sj;
        cr[threadIdx.x] = a;
        ci[threadIdx.x] = b;
        const float ah = (float)a, bh = (float)b;
        c4[threadIdx.x] = make_float4(ah, (float)(a - (double)ah), bh, (float)(b - (double)bh));
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kVecThreads) {
        CombineAcc<R> acc;
        for (int j = 0; j < m; ++j) acc.add(c4[j], cr[j], ci[j], V[(int64_t)j * n + i]);
        const auto o = acc.get();
        typename Cx<R>::T r;
        r.x = (R)o.x;
        r.y = (R)o.y;
        psi[i] = r;
    }
}

// k_reduce of apply.cu for the [nparts][4] partials (fixed order)
// beta_out (nullable): also sqrt(result[0]), the norm the sum of squares gives
__global__ void __launch_bounds__(1024) k_reduce4(const double *partials, int64_t nparts, double *result,
                                                  double *beta_out = nullptr) {
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
    if (t == 0 && beta_out) *beta_out = sqrt(sm[0][0]);
}

}  // namespace
}  // namespace ps

using namespace ps;

struct pauli_krylov {
    uint32_t magic;
    Allocator al;
    pauli_sum *H;
    const pauli_sector *s;
    int m, dtype;
    int64_t dim;
    void *V = nullptr;            // [m+1][dim] Lanczos vectors (v_m is scratch for w)
    KrylovScalars *sc = nullptr;  // device scalars
    double *partials = nullptr;   // vector-kernel partial sums
    int vec_blocks = 0;
    cudaGraphExec_t graph = nullptr;
    void *graph_psi = nullptr;
    double graph_dt = 0.0;
    // graphs are captured and replayed on a private stream ordered after / before
    // the caller's stream with events (the legacy default stream cannot capture)
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {
constexpr uint32_t kKrylovMagic = 0x504b5231u;

template <typename R>
void krylov_step_t(pauli_krylov *k, void *psi_v, double dt, cudaStream_t st) {
    using C2 = typename Cx<R>::T;
    C2 *psi = static_cast<C2 *>(psi_v);
    C2 *V = static_cast<C2 *>(k->V);
    const int64_t n = k->dim;
    const int nb = k->vec_blocks;
    Plan *p = find_plan(k->H, k->s->v);
    PS_CHECK(p != nullptr, PAULI_EINVAL, "krylov: operator plan missing");
    double *red = k->sc->red;
    // v_0 = psi / ||psi||
    k_norm2<R><<<nb, kVecThreads, 0, st>>>(psi, n, k->partials);
    k_reduce4<<<1, 1024, 0, st>>>(k->partials, nb, red);
    k_normalize<R><<<nb, kVecThreads, 0, st>>>(psi, V, n, k->sc, 0);
    PS_LAUNCH_CHECK();
    const int64_t nparts = apply_num_ctas(*p, k->s->v, k->dtype, true);
    PS_CHECK(p->partials != nullptr && nparts <= p->partials_cap, PAULI_EINVAL,
             "krylov: the plan's partial-sum buffer is too small (internal)");
    for (int j = 0; j < k->m; ++j) {
        C2 *vj = V + (int64_t)j * n;
        C2 *w = V + (int64_t)(j + 1) * n;  // w_j is built in place of v_{j+1}
        // w = H v_j with alpha_j = Re <v_j|H v_j> reduced in FP64
        launch_apply(k->H, *p, k->s->v, vj, w, k->dtype, p->partials, st, true);
        launch_reduce(p->partials, nparts, red, st);
        k_lanczos_update<R><<<nb, kVecThreads, 0, st>>>(w, vj, j > 0 ? V + (int64_t)(j - 1) * n : nullptr, n, k->sc,
                                                         j, k->partials);
        // beta_{j+1} = ||u_{j+1}||; u_{j+1} stays unnormalised (its scale enters the
        // next update and the combination)
        k_reduce4<<<1, 1024, 0, st>>>(k->partials, nb, red, k->sc->beta + j + 1);
        PS_LAUNCH_CHECK();
    }
    // beta_m of the last update is not needed by T_m; exp(-i dt T_m) e_0 and the combination
    k_tridiag_expm<<<1, 32, 0, st>>>(k->sc, k->m, dt);
    k_krylov_combine<R><<<nb, kVecThreads, 0, st>>>(V, n, k->m, k->sc, psi);
    PS_LAUNCH_CHECK();
}

void krylov_step(pauli_krylov *k, void *psi, double dt, cudaStream_t st) {
    if (k->dtype == PAULI_C64) krylov_step_t<float>(k, psi, dt, st);
    else krylov_step_t<double>(k, psi, dt, st);
}
}  // namespace

extern "C" {

int pauli_krylov_create(pauli_sum *H, const pauli_sector *s, int m, int dtype, pauli_krylov **out) {
    try {
        clear_error();
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(H && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(m >= 2 && m <= kMaxKrylov, PAULI_EINVAL, "m must be in 2..32");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(H->hermitian, PAULI_ENOTHERMITIAN, "Krylov propagation needs a Hermitian operator");
        int rc = pauli_prepare(H, s);
        if (rc != PAULI_OK) return rc;
        pauli_krylov *k = new pauli_krylov();
        k->magic = kKrylovMagic;
        k->al = current_allocator();
        k->H = H;
        k->s = s;
        k->m = m;
        k->dtype = dtype;
        k->dim = s->v.dim;
        try {
            const size_t es = dtype == PAULI_C64 ? 8 : 16;
            k->V = dev_alloc(k->al, (size_t)(m + 1) * (size_t)k->dim * es);
            k->sc = static_cast<KrylovScalars *>(dev_alloc(k->al, sizeof(KrylovScalars)));
            PS_CUDA(cudaMemset(k->sc, 0, sizeof(KrylovScalars)));
            int dev = 0, sms = 0;
            PS_CUDA(cudaGetDevice(&dev));
            PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            k->vec_blocks = sms * 8;
            k->partials = static_cast<double *>(dev_alloc(k->al, (size_t)k->vec_blocks * 4 * sizeof(double)));
            PS_CUDA(cudaStreamCreateWithFlags(&k->gstream, cudaStreamNonBlocking));
            PS_CUDA(cudaEventCreateWithFlags(&k->ev_in, cudaEventDisableTiming));
            PS_CUDA(cudaEventCreateWithFlags(&k->ev_out, cudaEventDisableTiming));
        } catch (...) {
            if (k->gstream) (void)cudaStreamDestroy(k->gstream);
            if (k->ev_in) (void)cudaEventDestroy(k->ev_in);
            if (k->ev_out) (void)cudaEventDestroy(k->ev_out);
            dev_free(k->al, k->V);
            dev_free(k->al, k->sc);
            dev_free(k->al, k->partials);
            delete k;
            throw;
        }
        *out = k;
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_krylov_step(pauli_krylov *k, void *psi, double dt, int nsteps, int use_graph, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(k && k->magic == kKrylovMagic, PAULI_EINVAL, "not a valid pauli_krylov handle");
        PS_CHECK(psi != nullptr && ((uintptr_t)psi % 16) == 0, PAULI_EINVAL, "psi is NULL or not 16-byte aligned");
        PS_CHECK(std::isfinite(dt), PAULI_EINVAL, "dt must be finite");
        PS_CHECK(nsteps >= 0, PAULI_EINVAL, "nsteps must be >= 0");
        cudaStream_t cs = (cudaStream_t)st;
        if (!use_graph) {
            for (int i = 0; i < nsteps; ++i) krylov_step(k, psi, dt, cs);
            return PAULI_OK;
        }
        if (nsteps == 0) return PAULI_OK;
        cudaStream_t gs = k->gstream;
        PS_CUDA(cudaEventRecord(k->ev_in, cs));
        PS_CUDA(cudaStreamWaitEvent(gs, k->ev_in, 0));
        if (!k->graph || k->graph_psi != psi || k->graph_dt != dt) {
            if (k->graph) {
                PS_CUDA(cudaGraphExecDestroy(k->graph));
                k->graph = nullptr;
            }
            // one eager step first: every kernel attribute is set outside the capture
            krylov_step(k, psi, dt, gs);
            --nsteps;
            cudaGraph_t g = nullptr;
            PS_CUDA(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal));
            try {
                krylov_step(k, psi, dt, gs);
            } catch (...) {
                cudaGraph_t dummy = nullptr;
                (void)cudaStreamEndCapture(gs, &dummy);
                if (dummy) (void)cudaGraphDestroy(dummy);
                throw;
            }
            PS_CUDA(cudaStreamEndCapture(gs, &g));
            cudaError_t e = cudaGraphInstantiate(&k->graph, g, 0);
            (void)cudaGraphDestroy(g);
            PS_CUDA(e);
            k->graph_psi = psi;
            k->graph_dt = dt;
        }
        for (int i = 0; i < nsteps; ++i) PS_CUDA(cudaGraphLaunch(k->graph, gs));
        PS_CUDA(cudaEventRecord(k->ev_out, gs));
        PS_CUDA(cudaStreamWaitEvent(cs, k->ev_out, 0));
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_krylov_scalars(const pauli_krylov *k, double *alpha, double *beta, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(k && k->magic == kKrylovMagic, PAULI_EINVAL, "not a valid pauli_krylov handle");
        PS_CHECK(alpha && beta, PAULI_EINVAL, "alpha / beta are NULL");
        KrylovScalars h;
        PS_CUDA(cudaMemcpyAsync(&h, k->sc, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)st));
        PS_CUDA(cudaStreamSynchronize((cudaStream_t)st));
        for (int j = 0; j < k->m; ++j) alpha[j] = h.alpha[j];
        for (int j = 0; j <= k->m; ++j) beta[j] = h.beta[j];
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

int pauli_krylov_destroy(pauli_krylov *k) {
    if (!k) return PAULI_OK;
    if (k->magic != kKrylovMagic) {
        set_error("not a valid pauli_krylov handle");
        return PAULI_EINVAL;
    }
    if (k->gstream) (void)cudaStreamSynchronize(k->gstream);
    if (k->graph) (void)cudaGraphExecDestroy(k->graph);
    if (k->gstream) (void)cudaStreamDestroy(k->gstream);
    if (k->ev_in) (void)cudaEventDestroy(k->ev_in);
    if (k->ev_out) (void)cudaEventDestroy(k->ev_out);
    dev_free(k->al, k->V);
    dev_free(k->al, k->sc);
    dev_free(k->al, k->partials);
    k->magic = 0;
    delete k;
    return PAULI_OK;
}

}  // extern "C"
