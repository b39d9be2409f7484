// linalg.cu -- vector primitives the variational drivers need on the device:
// FP64-accumulated inner products <x|y> and sequences of group rotations.
#include <cmath>
#include <vector>

#include "apply_kernels.cuh"

namespace ps {
namespace {

constexpr int kDotThreads = 256;

// partial sums of <x|y> = sum conj(x_i) y_i (per-thread DotAcc, FP64 across threads)
template <typename R>
__global__ void __launch_bounds__(kDotThreads) k_vdot(const typename Cx<R>::T *__restrict__ x,
                                                      const typename Cx<R>::T *__restrict__ y, int64_t n,
                                                      double *partials) {
    DotAcc<R> dot;
    for (int64_t i = (int64_t)blockIdx.x * kDotThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDotThreads)
        dot.add(x[i], y[i]);
    double re = dot.get_re(), im = dot.get_im();
    __shared__ double red[2][kDotThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = re;
        red[1][threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < kDotThreads / 32; ++w) s += red[threadIdx.x][w];
        partials[(int64_t)blockIdx.x * 4 + threadIdx.x] = s;
        partials[(int64_t)blockIdx.x * 4 + 2 + threadIdx.x] = 0.0;
    }
}

__global__ void __launch_bounds__(1024) k_reduce2(const double *partials, int64_t nparts, double *result) {
    __shared__ double sm[2][1024];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t i = t; i < nparts; i += 1024) {
        s0 += partials[i * 4];
        s1 += partials[i * 4 + 1];
    }
    sm[0][t] = s0;
    sm[1][t] = s1;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (t < o) {
            sm[0][t] += sm[0][t + o];
            sm[1][t] += sm[1][t + o];
        }
        __syncthreads();
    }
    if (t < 2) result[t] = sm[t][0];
}

DotScratch g_dot[64];

}  // namespace

// 8 blocks per SM: enough resident warps to stream at full bandwidth
DotScratch &dot_scratch() {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CHECK(dev >= 0 && dev < 64, PAULI_EUNSUPPORTED, "device ordinal out of range");
    DotScratch &d = g_dot[dev];
    if (!d.partials) {
        int sms = 0;
        PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        d.partials = static_cast<double *>(dev_alloc(Allocator(), (size_t)sms * 8 * 4 * sizeof(double)));
        d.blocks = sms * 8;
    }
    return d;
}

void launch_reduce2(const double *partials, int64_t nparts, double *result, cudaStream_t st) {
    k_reduce2<<<1, 1024, 0, st>>>(partials, nparts, result);
    PS_LAUNCH_CHECK();
}

}  // namespace ps

using namespace ps;

extern "C" {

int pauli_vdot(const void *x, const void *y, int64_t n, int dtype, double *result, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(result != nullptr, PAULI_EINVAL, "result must not be NULL");
        PS_CHECK(n >= 0, PAULI_EINVAL, "n must be >= 0");
        PS_CHECK(n == 0 || (x && y), PAULI_EINVAL, "x and y must not be NULL");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        PS_CHECK(((uintptr_t)x % 16) == 0 && ((uintptr_t)y % 16) == 0, PAULI_EINVAL, "x / y not 16-byte aligned");
        cudaStream_t cs = (cudaStream_t)st;
        DotScratch &d = dot_scratch();
        if (dtype == PAULI_C64)
            k_vdot<float><<<d.blocks, kDotThreads, 0, cs>>>(static_cast<const float2 *>(x), static_cast<const float2 *>(y), n,
                                                            d.partials);
        else
            k_vdot<double><<<d.blocks, kDotThreads, 0, cs>>>(static_cast<const double2 *>(x),
                                                             static_cast<const double2 *>(y), n, d.partials);
        PS_LAUNCH_CHECK();
        launch_reduce2(d.partials, d.blocks, result, cs);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_rotate_seq(pauli_sum *const *Gs, const double *thetas, int k, const pauli_sector *s, void *psi,
                     int dtype, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(k >= 0, PAULI_EINVAL, "k must be >= 0");
        PS_CHECK(k == 0 || (Gs && thetas), PAULI_EINVAL, "Gs / thetas must not be NULL");
        for (int j = 0; j < k; ++j) {
            const int rc = pauli_rotate(Gs[j], s, thetas[j], psi, dtype, st);
            if (rc != PAULI_OK) return rc;
        }
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

}  // extern "C"
