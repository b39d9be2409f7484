// mlp.cu -- the learned warm start: a small MLP  x -> tanh(x W1 + b1) ->
// tanh(. W2 + b2) -> . W3 + b3  trained by Adam on an MSE loss.  The two
// wide layers run on the tensor cores in BF16 with FP32 accumulation
// (mma.sync m16n8k16); master weights, biases, the first layer, the loss and
// Adam are FP32.  With batches of at most a few dozen points the GEMMs are
// 48 x 256 x 256 at most, far too small for a tcgen05/TMEM pipeline to pay
// for its setup, so each warp computes one 16 x 8 output tile from operands
// read straight from global memory (L1/L2-resident).
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ps_internal.cuh"

namespace ps {
namespace {

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t *>(&v);
}

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n], then tanh if act), A(m,k) =
// A[m*sa0 + k*sa1], B(k,n) = B[k*sb0 + n*sb1] (BF16); zero-padded edges.
// Writes the FP32 result to C (ldc) and, if Cb != null, a BF16 copy.
__global__ void k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int64_t sa0, int64_t sa1,
                            const __nv_bfloat16 *__restrict__ B, int64_t sb0, int64_t sb1, const float *__restrict__ bias,
                            int act, float *__restrict__ Cf, __nv_bfloat16 *__restrict__ Cb, int ldc) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    const int n0 = blockIdx.x * 8, m0 = blockIdx.y * 16;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    auto a_at = [&](int m, int k) { return (m < M && k < K) ? A[(int64_t)m * sa0 + (int64_t)k * sa1] : zero; };
    auto b_at = [&](int k, int n) { return (k < K && n < N) ? B[(int64_t)k * sb0 + (int64_t)n * sb1] : zero; };
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int ka = k0 + tg * 2;
        const uint32_t a0 = pack_bf16(a_at(m0 + g, ka), a_at(m0 + g, ka + 1));
        const uint32_t a1 = pack_bf16(a_at(m0 + g + 8, ka), a_at(m0 + g + 8, ka + 1));
        const uint32_t a2 = pack_bf16(a_at(m0 + g, ka + 8), a_at(m0 + g, ka + 9));
        const uint32_t a3 = pack_bf16(a_at(m0 + g + 8, ka + 8), a_at(m0 + g + 8, ka + 9));
        const uint32_t b0 = pack_bf16(b_at(ka, n0 + g), b_at(ka + 1, n0 + g));
        const uint32_t b1 = pack_bf16(b_at(ka + 8, n0 + g), b_at(ka + 9, n0 + g));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + g + ((i >= 2) ? 8 : 0);
        const int n = n0 + tg * 2 + (i & 1);
        if (m >= M || n >= N) continue;
        float v = c[i];
        if (bias) v += bias[n];
        if (act) v = tanhf(v);
        if (Cf) Cf[(int64_t)m * ldc + n] = v;
        if (Cb) Cb[(int64_t)m * ldc + n] = __float2bfloat16(v);
    }
}

// first layer: H1 = tanh(x W1 + b1), FP32 (+ BF16 copy)
__global__ void k_layer1(int B, int in, int hid, const float *x, const float *W1, const float *b1, float *H1,
                         __nv_bfloat16 *H1b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * hid) return;
    const int b = i / hid, j = i % hid;
    float z = b1[j];
    for (int k = 0; k < in; ++k) z += x[b * in + k] * W1[k * hid + j];
    const float h = tanhf(z);
    H1[i] = h;
    H1b[i] = __float2bfloat16(h);
}

// dY = (Y - T) / B (FP32 + BF16), loss partial sums per row
__global__ void k_mse_grad(int B, int out, const float *Y, const float *T, float *dY, __nv_bfloat16 *dYb,
                           double *loss_rows) {
    const int b = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < out; j += blockDim.x) {
        const float d = Y[b * out + j] - T[b * out + j];
        acc += (double)d * d;
        const float g = d / (float)B;
        dY[b * out + j] = g;
        dYb[b * out + j] = __float2bfloat16(g);
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_rows[b] = red[0];
}

__global__ void k_loss_sum(int B, const double *rows, double *loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < B; ++b) s += rows[b];
        *loss = 0.5 * s / B;
    }
}

// dZ = dH * (1 - H^2) (FP32 + BF16)
__global__ void k_tanh_back(int n, const float *dH, const float *H, float *dZ, __nv_bfloat16 *dZb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = dH[i] * (1.0f - H[i] * H[i]);
    dZ[i] = v;
    if (dZb) dZb[i] = __float2bfloat16(v);
}

// db[j] = sum_b dZ[b][j] (fixed order)
__global__ void k_colsum(int B, int n, const float *dZ, float *db) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += dZ[b * n + j];
    db[j] = s;
}

// dW1[k][j] = sum_b x[b][k] dZ1[b][j]
__global__ void k_dw1(int B, int in, int hid, const float *x, const float *dZ1, float *dW1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= in * hid) return;
    const int k = i / hid, j = i % hid;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += x[b * in + k] * dZ1[b * hid + j];
    dW1[i] = s;
}

__global__ void k_adam(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Adam with the bias corrections of the step (*step) of this training call taken
// from a host-computed table c12 = {1 - b1^t, 1 - b2^t} per step (the same float
// values as the eagerly launched k_adam gets), for the replayed graph of one step
__global__ void k_adam_tab(int64_t n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2,
                           float eps, const float *c12, const int *step) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = *step;
    const float c1 = c12[2 * s], c2 = c12[2 * s + 1];
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_step_inc(int *step) { ++*step; }

__global__ void k_to_bf16(int64_t n, const float *src, __nv_bfloat16 *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16(src[i]);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace ps

using namespace ps;

struct pauli_mlp {
    uint32_t magic;
    Allocator al;
    int in, hid, out, maxb;
    int64_t np;                // parameters
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // [np] each
    __nv_bfloat16 *W2b = nullptr, *W3b = nullptr;
    float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH2 = nullptr, *dZ2 = nullptr, *dH1 = nullptr,
          *dZ1 = nullptr;
    __nv_bfloat16 *H1b = nullptr, *H2b = nullptr, *dYb = nullptr, *dZ2b = nullptr;
    double *loss_rows = nullptr;
    // one training step captured as a CUDA graph and replayed (pauli_mlp_train):
    // the graph is keyed by the batch, the input / target pointers and lr
    cudaGraphExec_t gexec = nullptr;
    int g_batch = 0;
    const float *g_x = nullptr, *g_t = nullptr;
    float g_lr = 0.f;
    float *c12 = nullptr;      // [c12_cap][2] bias corrections of the call's steps (device)
    int c12_cap = 0;
    int *d_step = nullptr;     // the step being replayed (device)
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

namespace {
constexpr uint32_t kMlpMagic = 0x504d4c31u;

void mlp_forward(pauli_mlp *p, int B, const float *x, cudaStream_t st) {
    k_layer1<<<nb((int64_t)B * p->hid), 256, 0, st>>>(B, p->in, p->hid, x, p->w + p->oW1, p->w + p->ob1, p->H1, p->H1b);
    // H2 = tanh(H1 W2 + b2)
    dim3 g2((p->hid + 7) / 8, (B + 15) / 16);
    k_gemm_bf16<<<g2, 32, 0, st>>>(B, p->hid, p->hid, p->H1b, p->hid, 1, p->W2b, p->hid, 1, p->w + p->ob2, 1, p->H2,
                                   p->H2b, p->hid);
    // Y = H2 W3 + b3
    dim3 g3((p->out + 7) / 8, (B + 15) / 16);
    k_gemm_bf16<<<g3, 32, 0, st>>>(B, p->out, p->hid, p->H2b, p->hid, 1, p->W3b, p->out, 1, p->w + p->ob3, 0, p->Y,
                                   nullptr, p->out);
    PS_LAUNCH_CHECK();
}

void mlp_refresh_bf16(pauli_mlp *p, cudaStream_t st) {
    k_to_bf16<<<nb((int64_t)p->hid * p->hid), 256, 0, st>>>((int64_t)p->hid * p->hid, p->w + p->oW2, p->W2b);
    k_to_bf16<<<nb((int64_t)p->hid * p->out), 256, 0, st>>>((int64_t)p->hid * p->out, p->w + p->oW3, p->W3b);
    PS_LAUNCH_CHECK();
}

void mlp_backward(pauli_mlp *p, int batch, const float *x, const float *target, double *loss, cudaStream_t cs) {
    const int B = batch, H = p->hid, O = p->out;
    mlp_forward(p, B, x, cs);
    k_mse_grad<<<B, 256, 0, cs>>>(B, O, p->Y, target, p->dY, p->dYb, p->loss_rows);
    if (loss) k_loss_sum<<<1, 32, 0, cs>>>(B, p->loss_rows, loss);
    // dW3 = H2^T dY, db3 = colsum(dY)
    k_gemm_bf16<<<dim3((O + 7) / 8, (H + 15) / 16), 32, 0, cs>>>(H, O, B, p->H2b, 1, H, p->dYb, O, 1, nullptr, 0,
                                                               p->g + p->oW3, nullptr, O);
    k_colsum<<<nb(O), 256, 0, cs>>>(B, O, p->dY, p->g + p->ob3);
    // dH2 = dY W3^T ; dZ2 = dH2 (1 - H2^2)
    k_gemm_bf16<<<dim3((H + 7) / 8, (B + 15) / 16), 32, 0, cs>>>(B, H, O, p->dYb, O, 1, p->W3b, 1, O, nullptr, 0,
                                                               p->dH2, nullptr, H);
    k_tanh_back<<<nb((int64_t)B * H), 256, 0, cs>>>(B * H, p->dH2, p->H2, p->dZ2, p->dZ2b);
    // dW2 = H1^T dZ2, db2 = colsum(dZ2)
    k_gemm_bf16<<<dim3((H + 7) / 8, (H + 15) / 16), 32, 0, cs>>>(H, H, B, p->H1b, 1, H, p->dZ2b, H, 1, nullptr, 0,
                                                               p->g + p->oW2, nullptr, H);
    k_colsum<<<nb(H), 256, 0, cs>>>(B, H, p->dZ2, p->g + p->ob2);
    // dH1 = dZ2 W2^T ; dZ1 = dH1 (1 - H1^2)
    k_gemm_bf16<<<dim3((H + 7) / 8, (B + 15) / 16), 32, 0, cs>>>(B, H, H, p->dZ2b, H, 1, p->W2b, 1, H, nullptr, 0,
                                                               p->dH1, nullptr, H);
    k_tanh_back<<<nb((int64_t)B * H), 256, 0, cs>>>(B * H, p->dH1, p->H1, p->dZ1, nullptr);
    // dW1 = x^T dZ1, db1 = colsum(dZ1)
    k_dw1<<<nb((int64_t)p->in * H), 256, 0, cs>>>(B, p->in, H, x, p->dZ1, p->g + p->oW1);
    k_colsum<<<nb(H), 256, 0, cs>>>(B, H, p->dZ1, p->g + p->ob1);
    PS_LAUNCH_CHECK();
}

constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;

void adam_corrections(int t, float &c1, float &c2) {
    c1 = 1.f - std::pow(kAdamB1, (float)t);
    c2 = 1.f - std::pow(kAdamB2, (float)t);
}

void mlp_adam(pauli_mlp *p, float lr, int t, cudaStream_t cs) {
    float c1, c2;
    adam_corrections(t, c1, c2);
    k_adam<<<nb(p->np), 256, 0, cs>>>(p->np, p->w, p->g, p->m, p->v, lr, kAdamB1, kAdamB2, kAdamEps, c1, c2);
    PS_LAUNCH_CHECK();
    mlp_refresh_bf16(p, cs);
}

void free_train_graph(pauli_mlp *p) {
    if (p->gexec) (void)cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
}

// One step (forward, backward, Adam from the table, bf16 refresh, step counter)
// captured on the private stream; replayed steps - 1 times by pauli_mlp_train.
void capture_train_step(pauli_mlp *p, int batch, const float *x, const float *target, float lr) {
    free_train_graph(p);
    cudaGraph_t graph = nullptr;
    PS_CUDA(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    try {
        mlp_backward(p, batch, x, target, nullptr, p->gstream);
        k_adam_tab<<<nb(p->np), 256, 0, p->gstream>>>(p->np, p->w, p->g, p->m, p->v, lr, kAdamB1, kAdamB2, kAdamEps,
                                                      p->c12, p->d_step);
        mlp_refresh_bf16(p, p->gstream);
        k_step_inc<<<1, 1, 0, p->gstream>>>(p->d_step);
    } catch (...) {
        cudaGraph_t g = nullptr;
        (void)cudaStreamEndCapture(p->gstream, &g);
        if (g) (void)cudaGraphDestroy(g);
        throw;
    }
    PS_CUDA(cudaStreamEndCapture(p->gstream, &graph));
    cudaError_t e = cudaGraphInstantiate(&p->gexec, graph, 0);
    (void)cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        p->gexec = nullptr;
        throw Error{PAULI_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
    }
    p->g_batch = batch;
    p->g_x = x;
    p->g_t = target;
    p->g_lr = lr;
}

template <typename F>
int guard_mlp(F &&f) {
    try {
        clear_error();
        f();
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

void check_mlp(const pauli_mlp *p) {
    PS_CHECK(p != nullptr && p->magic == kMlpMagic, PAULI_EINVAL, "not a valid pauli_mlp handle");
}
}  // namespace

extern "C" {

int pauli_mlp_create(int in_dim, int hidden, int out_dim, int max_batch, pauli_mlp **out) {
    return guard_mlp([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(in_dim >= 1 && in_dim <= 64 && hidden >= 8 && hidden <= 4096 && out_dim >= 1 && out_dim <= 4096,
                 PAULI_EINVAL, "bad layer sizes");
        PS_CHECK(max_batch >= 1 && max_batch <= 65536, PAULI_EINVAL, "bad max_batch");
        pauli_mlp *p = new pauli_mlp();
        p->magic = kMlpMagic;
        p->al = current_allocator();
        p->in = in_dim;
        p->hid = hidden;
        p->out = out_dim;
        p->maxb = max_batch;
        p->oW1 = 0;
        p->ob1 = p->oW1 + (int64_t)in_dim * hidden;
        p->oW2 = p->ob1 + hidden;
        p->ob2 = p->oW2 + (int64_t)hidden * hidden;
        p->oW3 = p->ob2 + hidden;
        p->ob3 = p->oW3 + (int64_t)hidden * out_dim;
        p->np = p->ob3 + out_dim;
        try {
            auto f32 = [&](int64_t n) { return static_cast<float *>(dev_alloc(p->al, (size_t)n * sizeof(float))); };
            auto b16 = [&](int64_t n) {
                return static_cast<__nv_bfloat16 *>(dev_alloc(p->al, (size_t)n * sizeof(__nv_bfloat16)));
            };
            p->w = f32(p->np);
            p->g = f32(p->np);
            p->m = f32(p->np);
            p->v = f32(p->np);
            PS_CUDA(cudaMemset(p->w, 0, p->np * sizeof(float)));
            PS_CUDA(cudaMemset(p->m, 0, p->np * sizeof(float)));
            PS_CUDA(cudaMemset(p->v, 0, p->np * sizeof(float)));
            p->W2b = b16((int64_t)hidden * hidden);
            p->W3b = b16((int64_t)hidden * out_dim);
            const int64_t bh = (int64_t)max_batch * hidden, bo = (int64_t)max_batch * out_dim;
            p->H1 = f32(bh);
            p->H2 = f32(bh);
            p->Y = f32(bo);
            p->dY = f32(bo);
            p->dH2 = f32(bh);
            p->dZ2 = f32(bh);
            p->dH1 = f32(bh);
            p->dZ1 = f32(bh);
            p->H1b = b16(bh);
            p->H2b = b16(bh);
            p->dYb = b16(bo);
            p->dZ2b = b16(bh);
            p->loss_rows = static_cast<double *>(dev_alloc(p->al, (size_t)max_batch * sizeof(double)));
            mlp_refresh_bf16(p, nullptr);
            PS_CUDA(cudaDeviceSynchronize());
        } catch (...) {
            pauli_mlp_destroy(p);
            throw;
        }
        *out = p;
    });
}

int pauli_mlp_num_params(const pauli_mlp *p, int64_t *n) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(n != nullptr, PAULI_EINVAL, "n is NULL");
        *n = p->np;
    });
}

int pauli_mlp_set_params(pauli_mlp *p, const float *params) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(params != nullptr, PAULI_EINVAL, "params is NULL");
        PS_CUDA(cudaMemcpy(p->w, params, p->np * sizeof(float), cudaMemcpyHostToDevice));
        PS_CUDA(cudaMemset(p->m, 0, p->np * sizeof(float)));
        PS_CUDA(cudaMemset(p->v, 0, p->np * sizeof(float)));
        mlp_refresh_bf16(p, nullptr);
        PS_CUDA(cudaDeviceSynchronize());
    });
}

int pauli_mlp_get_params(const pauli_mlp *p, float *params) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(params != nullptr, PAULI_EINVAL, "params is NULL");
        PS_CUDA(cudaMemcpy(params, p->w, p->np * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

int pauli_mlp_forward(pauli_mlp *p, int batch, const float *x, float *y, pauli_stream_t st) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(batch >= 1 && batch <= p->maxb, PAULI_EINVAL, "batch out of range");
        PS_CHECK(x && y, PAULI_EINVAL, "x / y are NULL");
        cudaStream_t cs = (cudaStream_t)st;
        mlp_forward(p, batch, x, cs);
        PS_CUDA(cudaMemcpyAsync(y, p->Y, (size_t)batch * p->out * sizeof(float), cudaMemcpyDeviceToDevice, cs));
    });
}

int pauli_mlp_backward(pauli_mlp *p, int batch, const float *x, const float *target, float *grads, double *loss,
                       pauli_stream_t st) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(batch >= 1 && batch <= p->maxb, PAULI_EINVAL, "batch out of range");
        PS_CHECK(x && target, PAULI_EINVAL, "x / target are NULL");
        cudaStream_t cs = (cudaStream_t)st;
        mlp_backward(p, batch, x, target, loss, cs);
        if (grads) PS_CUDA(cudaMemcpyAsync(grads, p->g, p->np * sizeof(float), cudaMemcpyDeviceToDevice, cs));
    });
}

int pauli_mlp_adam_step(pauli_mlp *p, float lr, int t, pauli_stream_t st) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(t >= 1, PAULI_EINVAL, "t must be >= 1");
        PS_CHECK(std::isfinite(lr) && lr > 0.f, PAULI_EINVAL, "lr must be positive");
        mlp_adam(p, lr, t, (cudaStream_t)st);
    });
}

int pauli_mlp_train(pauli_mlp *p, int batch, const float *x, const float *target, int steps, float lr, int t0,
                    double *loss, pauli_stream_t st) {
    return guard_mlp([&] {
        check_mlp(p);
        PS_CHECK(batch >= 1 && batch <= p->maxb, PAULI_EINVAL, "batch out of range");
        PS_CHECK(x && target, PAULI_EINVAL, "x / target are NULL");
        PS_CHECK(steps >= 0 && t0 >= 0 && (int64_t)t0 + steps < (1ll << 30), PAULI_EINVAL, "bad steps / t0");
        PS_CHECK(std::isfinite(lr) && lr > 0.f, PAULI_EINVAL, "lr must be positive");
        cudaStream_t cs = (cudaStream_t)st;
        if (steps == 0) return;
        // the first steps - 1 steps replay a captured graph of one step on the private
        // stream, ordered after and before the caller's stream with events; the last
        // step runs eagerly (it also reduces the loss).  The arithmetic is that of the
        // eager steps: the same kernels, the same host-computed bias corrections.
        const int ng = steps - 1;
        if (ng > 0) {
            if (!p->gstream) {
                PS_CUDA(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
                PS_CUDA(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
                PS_CUDA(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
                p->d_step = static_cast<int *>(dev_alloc(p->al, sizeof(int)));
            }
            if (p->c12_cap < ng) {
                PS_CUDA(cudaStreamSynchronize(cs));
                PS_CUDA(cudaStreamSynchronize(p->gstream));
                free_train_graph(p);  // the graph holds the table's address
                dev_free(p->al, p->c12);
                p->c12 = nullptr;
                p->c12_cap = 0;
                p->c12 = static_cast<float *>(dev_alloc(p->al, (size_t)2 * ng * sizeof(float)));
                p->c12_cap = ng;
            }
            std::vector<float> c12((size_t)2 * ng);
            for (int s = 0; s < ng; ++s) adam_corrections(t0 + s + 1, c12[2 * s], c12[2 * s + 1]);
            PS_CUDA(cudaEventRecord(p->ev_in, cs));
            PS_CUDA(cudaStreamWaitEvent(p->gstream, p->ev_in, 0));
            // pageable sources: the copies are staged before they return
            PS_CUDA(cudaMemcpyAsync(p->c12, c12.data(), c12.size() * sizeof(float), cudaMemcpyHostToDevice,
                                    p->gstream));
            PS_CUDA(cudaMemsetAsync(p->d_step, 0, sizeof(int), p->gstream));
            if (!p->gexec || p->g_batch != batch || p->g_x != x || p->g_t != target || p->g_lr != lr)
                capture_train_step(p, batch, x, target, lr);
            for (int s = 0; s < ng; ++s) PS_CUDA(cudaGraphLaunch(p->gexec, p->gstream));
            PS_CUDA(cudaEventRecord(p->ev_out, p->gstream));
            PS_CUDA(cudaStreamWaitEvent(cs, p->ev_out, 0));
        }
        mlp_backward(p, batch, x, target, loss, cs);
        mlp_adam(p, lr, t0 + steps, cs);
    });
}

int pauli_mlp_destroy(pauli_mlp *p) {
    if (!p) return PAULI_OK;
    if (p->magic != kMlpMagic) {
        set_error("not a valid pauli_mlp handle");
        return PAULI_EINVAL;
    }
    if (p->gstream) (void)cudaStreamSynchronize(p->gstream);
    free_train_graph(p);
    if (p->gstream) (void)cudaStreamDestroy(p->gstream);
    if (p->ev_in) (void)cudaEventDestroy(p->ev_in);
    if (p->ev_out) (void)cudaEventDestroy(p->ev_out);
    void *bufs[] = {p->w, p->g, p->m, p->v, p->W2b, p->W3b, p->H1, p->H2, p->Y, p->dY, p->dH2, p->dZ2, p->dH1,
                    p->dZ1, p->H1b, p->H2b, p->dYb, p->dZ2b, p->loss_rows, p->c12, p->d_step};
    for (void *b : bufs) dev_free(p->al, b);
    p->magic = 0;
    delete p;
    return PAULI_OK;
}

}  // extern "C"
