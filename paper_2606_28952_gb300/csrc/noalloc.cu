// noalloc.cu -- pauli_expect_noalloc: the expectation value with its reduction
// scratch in a fixed static device array, so the call itself allocates nothing.
//
// pauli_expect keeps 4 doubles per thread block of partial sums in memory that
// the library allocates (on the first call for a sector, or in pauli_prepare).
// Some callers cannot have device memory allocated on their behalf: programs
// whose device memory is entirely owned by another allocator (a framework's
// caching pool sized to the whole GPU), and latency-critical loops where a
// cudaMalloc / cudaFree, which can synchronise the whole device, is not
// acceptable.  For them this entry point takes the partial sums from
// g_expect_scratch below instead.
#include <mutex>

#include "ps_internal.cuh"

namespace ps {
namespace {

// Thread blocks of one expectation launch the static scratch can hold
// (4 doubles each: 2 MiB per GPU that loads the library, kept until exit).
constexpr int64_t kNoallocMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

// The scratch.  Host code may not use this name as a device address: in host
// code it is a host-side stand-in.  Its device address is looked up once per
// device with cudaGetSymbolAddress (scratch_on_current_device below).
static __device__ __align__(256) double g_expect_scratch[kNoallocMaxBlocks * 4];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of g_expect_scratch on the current device (set-up on the
// first call for each device, with that device current).  The address is kept
// for the life of the process: it assumes that no cudaDeviceReset runs in
// between (a reset reloads the module and may move the array).
double *scratch_on_current_device() {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CHECK(dev >= 0 && dev < kMaxDevices, PAULI_EUNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        PS_CUDA(cudaGetSymbolAddress(&p, g_expect_scratch));
        PS_CHECK(p != nullptr, PAULI_ECUDA, "cudaGetSymbolAddress returned NULL for the expectation scratch");
        g_addr[dev] = static_cast<double *>(p);
    }
    return g_addr[dev];
}

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" int pauli_expect_noalloc(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype,
                                    double *result, void *hpsi_out, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(H != nullptr && H->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
        PS_CHECK(s != nullptr && s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "dtype must be PAULI_C64 or PAULI_C128");
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PS_CHECK(psi != nullptr && ((uintptr_t)psi % 16) == 0, PAULI_EINVAL, "psi is NULL or not 16-byte aligned");
        PS_CHECK(result != nullptr, PAULI_EINVAL, "result is NULL");
        const size_t bytes = (size_t)s->v.dim * (dtype == PAULI_C64 ? 8 : 16);
        if (hpsi_out) {
            PS_CHECK(((uintptr_t)hpsi_out % 16) == 0, PAULI_EINVAL, "hpsi_out is not 16-byte aligned");
            const char *a = static_cast<const char *>(psi);
            const char *b = static_cast<const char *>(hpsi_out);
            PS_CHECK(a + bytes <= b || b + bytes <= a, PAULI_EINVAL, "psi and hpsi_out overlap");
        }
        Plan *p = find_plan(H, s->v);
        PS_CHECK(p != nullptr, PAULI_EINVAL,
                 "no apply plan for this sector split: call pauli_prepare(H, s) once before pauli_expect_noalloc");
        // one CTA per (row, column tile), no split: the launch touches no scratch but the static array
        const int64_t nct = apply_num_ctas(*p, s->v, dtype, false);
        PS_CHECK(nct <= kNoallocMaxBlocks, PAULI_EUNSUPPORTED,
                 "pauli_expect_noalloc: this sector needs " + std::to_string(nct) +
                     " thread blocks of partial sums; the static scratch holds " + std::to_string(kNoallocMaxBlocks));
        // the full-space pass kernel accumulates H psi across its passes: without an
        // output vector it would use (and on first use allocate) the plan's own
        // dim-sized scratch, so that case needs hpsi_out or an existing scratch
        const ApplyCfg cfg = apply_config(*p, s->v, dtype, false);
        if (cfg.local && !hpsi_out)
            PS_CHECK(local_scratch_bytes(cfg.local_cl ? p->local_cl : p->local) >= (int64_t)bytes, PAULI_EUNSUPPORTED,
                     "pauli_expect_noalloc: this full-space operator is applied in passes that accumulate H psi in "
                     "a vector; pass hpsi_out (a dim-sized vector) or call pauli_expect once without it first");
        cudaStream_t cs = (cudaStream_t)st;
        if (nct == 0) {
            PS_CUDA(cudaMemsetAsync(result, 0, 4 * sizeof(double), cs));
            return PAULI_OK;
        }
        double *scratch = scratch_on_current_device();
        // every block overwrites its own 4 partials before k_reduce reads them,
        // so nothing left over from an earlier call has to be cleared
        launch_apply(H, *p, s->v, psi, hpsi_out, dtype, scratch, cs, false);
        launch_reduce(scratch, nct, result, cs);
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}
