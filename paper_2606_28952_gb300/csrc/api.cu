// api.cu -- the extern "C" entry points declared in include/paulisim.h.
//
// Each entry point validates its arguments on the host, converts failures into
// status codes (no exception crosses the ABI) and enqueues the kernels of
// build.cu, sector.cu and apply.cu.
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "ps_internal.cuh"

namespace ps {

namespace {
thread_local std::string g_err;
std::mutex g_alloc_mu;
Allocator g_alloc;
}  // namespace

void set_error(const std::string &msg) { g_err = msg; }
void clear_error() { g_err.clear(); }

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}
void set_current_allocator(const Allocator &a) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = a;
}

void *dev_alloc(const Allocator &a, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (a.alloc_fn) {
        p = a.alloc_fn(bytes, a.ctx);
        if (!p) throw Error{PAULI_ENOMEM, "device allocator returned NULL for " + std::to_string(bytes) + " bytes"};
        return p;
    }
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error{PAULI_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
    return p;
}

void dev_free(const Allocator &a, void *p) {
    if (!p) return;
    if (a.free_fn) a.free_fn(p, a.ctx);
    else (void)cudaFree(p);
}

void init_sector_view(SectorView &v, int n, int kind, int n_lo, int nb, const int *klo, const int *khi,
                      const int *qubit_irrep = nullptr);

// Raw entries of the operator product A B (eq. pauli_operator_multiplication,
// eq. pauli_prod_x / pauli_prod_z / pauli_prod_phase), entry k * mb + l for
// the pair (a_k, b_l):  x = xa ^ xb, z = za ^ zb,
//   (X^xa Z^za)(X^xb Z^zb) = (-1)^popcount(za & xb) X^x Z^z,
// so the XZ-form coefficient is Ca Cb (-1)^popcount(za & xb).  The complex
// product is formed as (ar br - ai bi, ar bi + ai br) with separately rounded
// products (no fused multiply-add); the sign is exact.
__global__ void k_sum_product(int64_t ma, const uint64_t *__restrict__ xa, const uint64_t *__restrict__ za,
                              const double2 *__restrict__ ca, int64_t mb, const uint64_t *__restrict__ xb,
                              const uint64_t *__restrict__ zb, const double2 *__restrict__ cb, uint64_t *ox,
                              uint64_t *oz, double2 *oc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ma * mb) return;
    const int64_t k = i / mb, l = i - k * mb;
    const uint64_t x1 = xa[k], z1 = za[k], x2 = xb[l], z2 = zb[l];
    const double2 a = ca[k], b = cb[l];
    const double rr = __dmul_rn(a.x, b.x), ii = __dmul_rn(a.y, b.y);
    const double ri = __dmul_rn(a.x, b.y), ir = __dmul_rn(a.y, b.x);
    double re = __dsub_rn(rr, ii), im = __dadd_rn(ri, ir);
    if (__popcll(z1 & x2) & 1) {
        re = -re;
        im = -im;
    }
    ox[i] = x1 ^ x2;
    oz[i] = z1 ^ z2;
    oc[i] = make_double2(re, im);
}

// Raw entries of A + beta B: A's terms, then B's with beta C (same product rule).
__global__ void k_sum_scaled_copy(int64_t m, const double2 *__restrict__ c, double br, double bi, double2 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double2 a = c[i];
    out[i] = make_double2(__dsub_rn(__dmul_rn(a.x, br), __dmul_rn(a.y, bi)),
                          __dadd_rn(__dmul_rn(a.x, bi), __dmul_rn(a.y, br)));
}


namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void *>, size_t> g_attr;  // (device, kernel) -> dynamic smem opted in
constexpr int kMaxDev = 64;
int g_sms[kMaxDev] = {};
}  // namespace

void smem_optin(const void *func, size_t bytes) {
    // without the opt-in a block gets 48 KB of shared memory, static and dynamic together
    if (bytes == 0) return;
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &have = g_attr[std::make_pair(dev, func)];
    if (have >= bytes) return;
    cudaFuncAttributes fa;
    PS_CUDA(cudaFuncGetAttributes(&fa, func));
    if (bytes + fa.sharedSizeBytes > 48 * 1024)
        PS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
}

int num_sms() {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < kMaxDev && g_sms[dev] > 0) return g_sms[dev];
    int sms = 0;
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < kMaxDev) g_sms[dev] = sms;
    return sms;
}

}  // namespace ps

using namespace ps;

namespace {

template <typename F>
int guarded(F &&f) {
    try {
        clear_error();
        f();
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return PAULI_ENOMEM;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

struct PrivateStream {
    cudaStream_t s = nullptr;
    PrivateStream() { PS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
    ~PrivateStream() {
        if (s) {
            (void)cudaStreamSynchronize(s);
            (void)cudaStreamDestroy(s);
        }
    }
};

void check_sum(const pauli_sum *h) {
    PS_CHECK(h != nullptr, PAULI_EINVAL, "pauli_sum handle is NULL");
    PS_CHECK(h->magic == kSumMagic, PAULI_EINVAL, "not a valid pauli_sum handle");
}
void check_sector(const pauli_sector *s) {
    PS_CHECK(s != nullptr, PAULI_EINVAL, "pauli_sector handle is NULL");
    PS_CHECK(s->magic == kSectorMagic, PAULI_EINVAL, "not a valid pauli_sector handle");
}
void check_dtype(int dtype) {
    PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "dtype must be PAULI_C64 or PAULI_C128");
}
size_t elem_size(int dtype) { return dtype == PAULI_C64 ? 8 : 16; }
void check_state_ptr(const void *p, int dtype, const char *name) {
    PS_CHECK(p != nullptr, PAULI_EINVAL, std::string(name) + " is NULL");
    PS_CHECK(((uintptr_t)p % 16) == 0, PAULI_EINVAL, std::string(name) + " is not 16-byte aligned");
}

pauli_sum *new_sum(int n) {
    pauli_sum *h = new pauli_sum();
    h->magic = kSumMagic;
    h->al = current_allocator();
    h->n = n;
    try {
        h->status = static_cast<int *>(dev_alloc(h->al, sizeof(int)));
        PS_CUDA(cudaMemset(h->status, 0, sizeof(int)));
    } catch (...) {
        delete h;
        throw;
    }
    return h;
}

void destroy_sum(pauli_sum *h) {
    if (!h) return;
    for (int i = 0; i < h->nplans; ++i) free_plan(h->al, h->plans[i]);
    for (int i = 0; i < h->nrot; ++i) dev_free(h->al, h->rot[i].tab);
    dev_free(h->al, h->leak_flag);
    dev_free(h->al, h->x);
    dev_free(h->al, h->z);
    dev_free(h->al, h->c);
    dev_free(h->al, h->gx);
    dev_free(h->al, h->gstart);
    dev_free(h->al, h->status);
    dev_free(h->al, h->rows_part);
    h->magic = 0;
    delete h;
}

struct SumGuard {
    pauli_sum *h;
    explicit SumGuard(pauli_sum *p) : h(p) {}
    ~SumGuard() { destroy_sum(h); }
    pauli_sum *release() { pauli_sum *p = h; h = nullptr; return p; }
};

void check_integrals(int norb, const double *h, const double *g) {
    PS_CHECK(norb >= 1 && norb <= 32, PAULI_EINVAL, "n_orb must be in 1..32");
    PS_CHECK(h && g, PAULI_EINVAL, "integral arrays must not be NULL");
    const int64_t n2 = (int64_t)norb * norb, n4 = n2 * n2;
    for (int64_t i = 0; i < n2; ++i) PS_CHECK(std::isfinite(h[i]), PAULI_EINVAL, "h has a non-finite entry");
    for (int64_t i = 0; i < n4; ++i) PS_CHECK(std::isfinite(g[i]), PAULI_EINVAL, "g has a non-finite entry");
}

Plan &ensure_plan(pauli_sum *H, const pauli_sector *s, cudaStream_t st, bool need_partials) {
    Plan &p = get_plan(H, s->v, st);
    prepare_for_sector(H, p, s->v, st);
    ensure_df_capacity(H, p, s->v, st);
    // partial vectors of split launches (the split count depends on the dtype:
    // sized for both, so that either precision can run on the same plan)
    const int64_t split_bytes = std::max(apply_split_elems(p, s->v, PAULI_C64) * 8,
                                         apply_split_elems(p, s->v, PAULI_C128) * 16);
    if (p.split_cap < split_bytes) {
        PS_CUDA(cudaStreamSynchronize(st));
        dev_free(H->al, p.split_buf);
        p.split_buf = nullptr;
        p.split_cap = 0;
        p.split_buf = dev_alloc(H->al, (size_t)split_bytes);
        p.split_cap = split_bytes;
    }
    if (need_partials) {
        // one 4-double slot per CTA that writes partials, for either precision (their
        // launch shapes differ, e.g. a split in complex64 only) and either split mode
        int64_t nct = 0;
        for (int dt : {PAULI_C64, PAULI_C128})
            for (bool split : {true, false}) nct = std::max(nct, apply_num_ctas(p, s->v, dt, split));
        if (p.partials_cap < nct) {
            PS_CUDA(cudaStreamSynchronize(st));
            dev_free(H->al, p.partials);
            p.partials = nullptr;
            p.partials_cap = 0;
            p.partials = static_cast<double *>(dev_alloc(H->al, (size_t)(nct > 0 ? nct : 1) * 4 * sizeof(double)));
            p.partials_cap = nct;
        }
    }
    return p;
}

}  // namespace

extern "C" {

int pauli_sum_product(const pauli_sum *A, const pauli_sum *B, double eps_drop, pauli_sum **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        check_sum(A);
        check_sum(B);
        PS_CHECK(A->n == B->n, PAULI_EINVAL, "operands have different qubit counts");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        const int64_t m = A->m * B->m;
        PS_CHECK(A->m == 0 || m / A->m == B->m, PAULI_EUNSUPPORTED, "product too large");
        PS_CHECK(m <= (1ll << 31), PAULI_EUNSUPPORTED,
                 "product: more than 2^31 raw term pairs (" + std::to_string(m) + ")");
        PrivateStream ps_;
        SumGuard g(new_sum(A->n));
        const Allocator &al = g.h->al;
        DevBuf<uint64_t> dx(al, m), dz(al, m);
        DevBuf<double2> dc(al, m);
        if (m > 0) {
            k_sum_product<<<(unsigned)((m + 255) / 256), 256, 0, ps_.s>>>(A->m, A->x, A->z, A->c, B->m, B->x, B->z,
                                                                          B->c, dx.p, dz.p, dc.p);
            PS_LAUNCH_CHECK();
        }
        canonicalize(g.h, m, dx.p, dz.p, dc.p, eps_drop, ps_.s);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
        *out = g.release();
    });
}

int pauli_sum_add(const pauli_sum *A, const pauli_sum *B, double beta_re, double beta_im, double eps_drop,
                  pauli_sum **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        check_sum(A);
        check_sum(B);
        PS_CHECK(A->n == B->n, PAULI_EINVAL, "operands have different qubit counts");
        PS_CHECK(std::isfinite(beta_re) && std::isfinite(beta_im), PAULI_EINVAL, "beta must be finite");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        const int64_t m = A->m + B->m;
        PrivateStream ps_;
        SumGuard g(new_sum(A->n));
        const Allocator &al = g.h->al;
        DevBuf<uint64_t> dx(al, m), dz(al, m);
        DevBuf<double2> dc(al, m);
        if (A->m > 0) {
            PS_CUDA(cudaMemcpyAsync(dx.p, A->x, A->m * 8, cudaMemcpyDeviceToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dz.p, A->z, A->m * 8, cudaMemcpyDeviceToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dc.p, A->c, A->m * 16, cudaMemcpyDeviceToDevice, ps_.s));
        }
        if (B->m > 0) {
            PS_CUDA(cudaMemcpyAsync(dx.p + A->m, B->x, B->m * 8, cudaMemcpyDeviceToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dz.p + A->m, B->z, B->m * 8, cudaMemcpyDeviceToDevice, ps_.s));
            k_sum_scaled_copy<<<(unsigned)((B->m + 255) / 256), 256, 0, ps_.s>>>(B->m, B->c, beta_re, beta_im,
                                                                                dc.p + A->m);
            PS_LAUNCH_CHECK();
        }
        canonicalize(g.h, m, dx.p, dz.p, dc.p, eps_drop, ps_.s);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
        *out = g.release();
    });
}

const char *pauli_last_error(void) { return g_err.c_str(); }

int pauli_version(void) { return 10000; }

int pauli_set_allocator(void *(*alloc_fn)(size_t, void *), void (*free_fn)(void *, void *), void *ctx) {
    return guarded([&] {
        PS_CHECK((alloc_fn == nullptr) == (free_fn == nullptr), PAULI_EINVAL,
                 "alloc_fn and free_fn must both be set or both be NULL");
        Allocator a;
        a.alloc_fn = alloc_fn;
        a.free_fn = free_fn;
        a.ctx = alloc_fn ? ctx : nullptr;
        set_current_allocator(a);
    });
}

int pauli_sum_build(int n_qubits, int64_t m, const uint64_t *x, const uint64_t *z, const uint8_t *gamma,
                    const double *c_re, const double *c_im, int coeff_form, double eps_drop,
                    pauli_sum **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n_qubits >= 1 && n_qubits <= 64, PAULI_EINVAL, "n_qubits must be in 1..64");
        PS_CHECK(m >= 0, PAULI_EINVAL, "m must be >= 0");
        PS_CHECK(m == 0 || (x && z && c_re && c_im), PAULI_EINVAL, "term arrays must not be NULL");
        PS_CHECK(coeff_form == PAULI_LETTER || coeff_form == PAULI_XZ, PAULI_EINVAL, "bad coeff_form");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        const uint64_t mask = n_qubits == 64 ? ~0ull : ((1ull << n_qubits) - 1ull);
        for (int64_t i = 0; i < m; ++i) {
            PS_CHECK(((x[i] | z[i]) & ~mask) == 0, PAULI_EINVAL,
                     "term " + std::to_string(i) + " has a mask bit at or above n_qubits");
            PS_CHECK(std::isfinite(c_re[i]) && std::isfinite(c_im[i]), PAULI_EINVAL,
                     "term " + std::to_string(i) + " has a non-finite coefficient");
        }
        PrivateStream ps_;
        SumGuard g(new_sum(n_qubits));
        const Allocator &al = g.h->al;
        DevBuf<uint64_t> dx(al, m), dz(al, m);
        DevBuf<double> dre(al, m), dim_(al, m);
        DevBuf<uint8_t> dg(al, gamma ? m : 0);
        DevBuf<double2> dc(al, m);
        if (m > 0) {
            PS_CUDA(cudaMemcpyAsync(dx.p, x, m * 8, cudaMemcpyHostToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dz.p, z, m * 8, cudaMemcpyHostToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dre.p, c_re, m * 8, cudaMemcpyHostToDevice, ps_.s));
            PS_CUDA(cudaMemcpyAsync(dim_.p, c_im, m * 8, cudaMemcpyHostToDevice, ps_.s));
            if (gamma) PS_CUDA(cudaMemcpyAsync(dg.p, gamma, m, cudaMemcpyHostToDevice, ps_.s));
            to_xz_device(m, dx.p, dz.p, gamma ? dg.p : nullptr, dre.p, dim_.p, coeff_form == PAULI_LETTER,
                         dc.p, ps_.s);
        }
        canonicalize(g.h, m, dx.p, dz.p, dc.p, eps_drop, ps_.s);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
        *out = g.release();
    });
}

int pauli_jw_molecular(int n_orb, const double *h, const double *g, double e_nn, double eps_int,
                       double eps_drop, pauli_sum **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        check_integrals(n_orb, h, g);
        PS_CHECK(std::isfinite(e_nn), PAULI_EINVAL, "e_nn must be finite");
        PS_CHECK(std::isfinite(eps_int) && eps_int >= 0.0, PAULI_EINVAL, "eps_int must be finite and >= 0");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        PrivateStream ps_;
        SumGuard sg(new_sum(2 * n_orb));
        DevBuf<uint64_t> x, z;
        DevBuf<double2> c;
        int64_t count = 0;
        jw_molecular_raw_device(n_orb, h, g, e_nn, eps_int, sg.h->al, x, z, c, count, ps_.s);
        canonicalize(sg.h, count, x.p, z.p, c.p, eps_drop, ps_.s);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
        *out = sg.release();
    });
}

int pauli_jw_molecular_raw(int n_orb, const double *h, const double *g, double e_nn, double eps_int,
                           int64_t *count, uint64_t *x, uint64_t *z, double *c_re, double *c_im) {
    return guarded([&] {
        PS_CHECK(count != nullptr, PAULI_EINVAL, "count is NULL");
        check_integrals(n_orb, h, g);
        PS_CHECK(x == nullptr || (z && c_re && c_im), PAULI_EINVAL, "output arrays must all be set");
        PrivateStream ps_;
        const Allocator al = current_allocator();
        DevBuf<uint64_t> dx, dz;
        DevBuf<double2> dc;
        int64_t n = 0;
        jw_molecular_raw_device(n_orb, h, g, e_nn, eps_int, al, dx, dz, dc, n, ps_.s);
        if (x) {
            PS_CHECK(*count >= n, PAULI_EINVAL, "output arrays too small (need " + std::to_string(n) + ")");
            std::vector<double2> hc(n);
            PS_CUDA(cudaMemcpy(x, dx.p, n * 8, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(z, dz.p, n * 8, cudaMemcpyDeviceToHost));
            PS_CUDA(cudaMemcpy(hc.data(), dc.p, n * 16, cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < n; ++i) {
                c_re[i] = hc[i].x;
                c_im[i] = hc[i].y;
            }
        }
        *count = n;
    });
}

int pauli_jw_fermion(int n_qubits, int n_terms, const int *n_factors, const int *modes, const int *daggers,
                     const double *c_re, const double *c_im, double eps_drop, pauli_sum **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n_qubits >= 1 && n_qubits <= 64, PAULI_EINVAL, "n_qubits must be in 1..64");
        PS_CHECK(n_terms >= 0, PAULI_EINVAL, "n_terms must be >= 0");
        PS_CHECK(n_terms == 0 || (n_factors && c_re && c_im), PAULI_EINVAL, "term arrays must not be NULL");
        PS_CHECK(std::isfinite(eps_drop) && eps_drop >= 0.0, PAULI_EINVAL, "eps_drop must be finite and >= 0");
        int nf_total = 0;
        for (int t = 0; t < n_terms; ++t) {
            PS_CHECK(n_factors[t] >= 1 && n_factors[t] <= 8, PAULI_EINVAL, "each term needs 1..8 factors");
            PS_CHECK(std::isfinite(c_re[t]) && std::isfinite(c_im[t]), PAULI_EINVAL, "non-finite coefficient");
            nf_total += n_factors[t];
        }
        PS_CHECK(nf_total == 0 || (modes && daggers), PAULI_EINVAL, "modes / daggers must not be NULL");
        for (int j = 0; j < nf_total; ++j)
            PS_CHECK(modes[j] >= 0 && modes[j] < n_qubits, PAULI_EINVAL, "mode index out of range");
        PrivateStream ps_;
        SumGuard sg(new_sum(n_qubits));
        DevBuf<uint64_t> x, z;
        DevBuf<double2> c;
        int64_t count = 0;
        if (n_terms > 0)
            jw_fermion_raw_device(n_qubits, n_terms, n_factors, modes, daggers, c_re, c_im, sg.h->al, x, z, c,
                                  count, ps_.s);
        canonicalize(sg.h, count, x.p, z.p, c.p, eps_drop, ps_.s);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
        *out = sg.release();
    });
}

int pauli_sum_info(const pauli_sum *h, int *n_qubits, int64_t *m, int64_t *n_groups) {
    return guarded([&] {
        check_sum(h);
        if (n_qubits) *n_qubits = h->n;
        if (m) *m = h->m;
        if (n_groups) *n_groups = h->G;
    });
}

int pauli_sum_export(const pauli_sum *h, uint64_t *x, uint64_t *z, double *c_re, double *c_im) {
    return guarded([&] {
        check_sum(h);
        if (h->m == 0) return;
        PS_CHECK(x && z && c_re && c_im, PAULI_EINVAL, "output arrays must not be NULL");
        std::vector<double2> hc(h->m);
        PS_CUDA(cudaMemcpy(x, h->x, h->m * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(z, h->z, h->m * 8, cudaMemcpyDeviceToHost));
        PS_CUDA(cudaMemcpy(hc.data(), h->c, h->m * 16, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < h->m; ++i) {
            c_re[i] = hc[i].x;
            c_im[i] = hc[i].y;
        }
    });
}

int pauli_sum_groups(const pauli_sum *h, uint64_t *group_x, int64_t *group_start) {
    return guarded([&] {
        check_sum(h);
        PS_CHECK(group_start != nullptr, PAULI_EINVAL, "group_start is NULL");
        PS_CUDA(cudaMemcpy(group_start, h->gstart, (h->G + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (h->G > 0) {
            PS_CHECK(group_x != nullptr, PAULI_EINVAL, "group_x is NULL");
            PS_CUDA(cudaMemcpy(group_x, h->gx, h->G * sizeof(uint64_t), cudaMemcpyDeviceToHost));
        }
    });
}

int pauli_sum_destroy(pauli_sum *h) {
    return guarded([&] {
        if (!h) return;
        check_sum(h);
        destroy_sum(h);
    });
}

int pauli_sector_create(int n_qubits, int kind, int n_lo, int n_blocks, const int *k_lo, const int *k_hi,
                        pauli_sector **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(kind == PAULI_SECTOR_FULL || kind == PAULI_SECTOR_BLOCKS, PAULI_EINVAL, "bad sector kind");
        if (kind == PAULI_SECTOR_FULL) {
            PS_CHECK(n_qubits >= 1 && n_qubits <= 40, PAULI_EINVAL, "FULL sectors need 1 <= n_qubits <= 40");
            if (n_lo == 0) n_lo = n_qubits < 10 ? n_qubits : 10;
            PS_CHECK(n_lo >= 1 && n_lo <= n_qubits && n_lo <= kMaxHalf, PAULI_EINVAL, "bad n_lo for FULL sector");
            PS_CHECK(n_qubits - n_lo <= 31, PAULI_EUNSUPPORTED, "FULL sector: n_qubits - n_lo must be <= 31");
        } else {
            PS_CHECK(n_qubits >= 2 && n_qubits <= 2 * kMaxHalf, PAULI_EINVAL, "BLOCKS sectors need 2 <= n_qubits <= 48");
            PS_CHECK(n_lo >= 1 && n_lo < n_qubits && n_lo <= kMaxHalf && n_qubits - n_lo <= kMaxHalf,
                     PAULI_EINVAL, "BLOCKS sector: need 1 <= n_lo < n_qubits and both halves <= 24 qubits");
            PS_CHECK(n_blocks >= 1 && n_blocks <= kMaxBlocks, PAULI_EINVAL, "need 1..33 blocks");
            PS_CHECK(k_lo && k_hi, PAULI_EINVAL, "k_lo / k_hi must not be NULL");
            bool seen[kMaxHalf + 1] = {};
            for (int r = 0; r < n_blocks; ++r) {
                PS_CHECK(k_lo[r] >= 0 && k_lo[r] <= n_lo, PAULI_EINVAL, "k_lo out of range");
                PS_CHECK(k_hi[r] >= 0 && k_hi[r] <= n_qubits - n_lo, PAULI_EINVAL, "k_hi out of range");
                PS_CHECK(!seen[k_hi[r]], PAULI_EINVAL, "the k_hi of the blocks must be distinct");
                seen[k_hi[r]] = true;
            }
        }
        pauli_sector *s = new pauli_sector();
        s->magic = kSectorMagic;
        static std::atomic<uint64_t> next_uid{1};
        s->uid = next_uid.fetch_add(1);
        s->al = current_allocator();
        try {
            init_sector_view(s->v, n_qubits, kind, n_lo, n_blocks, k_lo, k_hi);
            PrivateStream ps_;
            build_sector_tables(s, ps_.s);
        } catch (...) {
            dev_free(s->al, s->tables);
            delete s;
            throw;
        }
        *out = s;
    });
}

int pauli_sector_create_irrep(int n_qubits, int n_lo, int n_blocks, const int *k_lo, const int *irrep_lo,
                              const int *k_hi, const int *irrep_hi, const int *qubit_irrep, pauli_sector **out) {
    return guarded([&] {
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n_qubits >= 2 && n_qubits <= 2 * kMaxHalf, PAULI_EINVAL, "point-group sectors need 2 <= n_qubits <= 48");
        PS_CHECK(n_lo >= 1 && n_lo < n_qubits && n_lo <= kMaxHalf && n_qubits - n_lo <= kMaxHalf, PAULI_EINVAL,
                 "need 1 <= n_lo < n_qubits and both halves <= 24 qubits");
        PS_CHECK(n_blocks >= 1 && n_blocks <= kMaxBlocks, PAULI_EINVAL, "need 1..33 blocks");
        PS_CHECK(k_lo && k_hi && irrep_lo && irrep_hi && qubit_irrep, PAULI_EINVAL, "block / label arrays must not be NULL");
        for (int q = 0; q < n_qubits; ++q)
            PS_CHECK(qubit_irrep[q] >= 0 && qubit_irrep[q] <= 7, PAULI_EINVAL, "qubit irreps must be in 0..7");
        std::vector<int> klo(n_blocks), khi(n_blocks);
        bool seen[kMaxCls] = {};
        for (int r = 0; r < n_blocks; ++r) {
            PS_CHECK(k_lo[r] >= 0 && k_lo[r] <= n_lo && k_hi[r] >= 0 && k_hi[r] <= n_qubits - n_lo, PAULI_EINVAL,
                     "k_lo / k_hi out of range");
            PS_CHECK(irrep_lo[r] >= 0 && irrep_lo[r] <= 7 && irrep_hi[r] >= 0 && irrep_hi[r] <= 7, PAULI_EINVAL,
                     "block irreps must be in 0..7");
            klo[r] = k_lo[r] * 8 + irrep_lo[r];
            khi[r] = k_hi[r] * 8 + irrep_hi[r];
            PS_CHECK(!seen[khi[r]], PAULI_EINVAL, "the (k_hi, irrep_hi) of the blocks must be distinct");
            seen[khi[r]] = true;
        }
        pauli_sector *s = new pauli_sector();
        s->magic = kSectorMagic;
        static std::atomic<uint64_t> next_uid{1ull << 40};
        s->uid = next_uid.fetch_add(1);
        s->al = current_allocator();
        try {
            init_sector_view(s->v, n_qubits, PAULI_SECTOR_BLOCKS, n_lo, n_blocks, klo.data(), khi.data(), qubit_irrep);
            PrivateStream ps_;
            build_sector_tables(s, ps_.s);
        } catch (...) {
            dev_free(s->al, s->tables);
            delete s;
            throw;
        }
        *out = s;
    });
}

int pauli_sector_dim(const pauli_sector *s, int64_t *dim) {
    return guarded([&] {
        check_sector(s);
        PS_CHECK(dim != nullptr, PAULI_EINVAL, "dim is NULL");
        *dim = s->v.dim;
    });
}

int pauli_sector_rank(const pauli_sector *s, const uint64_t *configs, int64_t n, int64_t *idx, pauli_stream_t st) {
    return guarded([&] {
        check_sector(s);
        PS_CHECK(n >= 0, PAULI_EINVAL, "n must be >= 0");
        PS_CHECK(n == 0 || (configs && idx), PAULI_EINVAL, "arrays must not be NULL");
        sector_rank(s->v, configs, n, idx, (cudaStream_t)st);
    });
}

int pauli_sector_unrank(const pauli_sector *s, const int64_t *idx, int64_t n, uint64_t *configs, pauli_stream_t st) {
    return guarded([&] {
        check_sector(s);
        PS_CHECK(n >= 0, PAULI_EINVAL, "n must be >= 0");
        PS_CHECK(n == 0 || (configs && idx), PAULI_EINVAL, "arrays must not be NULL");
        sector_unrank(s->v, idx, n, configs, (cudaStream_t)st);
    });
}

int pauli_sector_destroy(pauli_sector *s) {
    return guarded([&] {
        if (!s) return;
        check_sector(s);
        dev_free(s->al, s->tables);
        s->magic = 0;
        delete s;
    });
}

int pauli_prepare(pauli_sum *H, const pauli_sector *s) {
    return guarded([&] {
        check_sum(H);
        check_sector(s);
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        PrivateStream ps_;
        ensure_plan(H, s, ps_.s, true);
        PS_CUDA(cudaStreamSynchronize(ps_.s));
    });
}

int pauli_apply(pauli_sum *H, const pauli_sector *s, const void *psi_in, void *psi_out, int dtype,
                pauli_stream_t st) {
    return guarded([&] {
        check_sum(H);
        check_sector(s);
        check_dtype(dtype);
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        check_state_ptr(psi_in, dtype, "psi_in");
        check_state_ptr(psi_out, dtype, "psi_out");
        const size_t bytes = (size_t)s->v.dim * elem_size(dtype);
        const char *a = static_cast<const char *>(psi_in);
        const char *b = static_cast<const char *>(psi_out);
        PS_CHECK(a + bytes <= b || b + bytes <= a, PAULI_EINVAL, "psi_in and psi_out overlap");
        cudaStream_t cs = (cudaStream_t)st;
        Plan &p = ensure_plan(H, s, cs, false);
        launch_apply(H, p, s->v, psi_in, psi_out, dtype, nullptr, cs);
    });
}

int pauli_expect(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype, double *result, void *hpsi_out,
                 pauli_stream_t st) {
    return guarded([&] {
        check_sum(H);
        check_sector(s);
        check_dtype(dtype);
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        check_state_ptr(psi, dtype, "psi");
        PS_CHECK(result != nullptr, PAULI_EINVAL, "result is NULL");
        if (hpsi_out) {
            check_state_ptr(hpsi_out, dtype, "hpsi_out");
            const size_t bytes = (size_t)s->v.dim * elem_size(dtype);
            const char *a = static_cast<const char *>(psi);
            const char *b = static_cast<const char *>(hpsi_out);
            PS_CHECK(a + bytes <= b || b + bytes <= a, PAULI_EINVAL, "psi and hpsi_out overlap");
        }
        cudaStream_t cs = (cudaStream_t)st;
        Plan &p = ensure_plan(H, s, cs, true);
        const int64_t nct = apply_num_ctas(p, s->v, dtype, true);
        if (nct == 0) {
            PS_CUDA(cudaMemsetAsync(result, 0, 4 * sizeof(double), cs));
            return;
        }
        PS_CHECK(p.partials != nullptr && nct <= p.partials_cap, PAULI_EINVAL,
                 "expect: the plan's partial-sum buffer is too small (internal)");
        launch_apply(H, p, s->v, psi, hpsi_out, dtype, p.partials, cs);
        launch_reduce(p.partials, nct, result, cs);
    });
}

int pauli_expect_rows(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype, const int64_t *rows,
                      int64_t n_rows, void *hpsi_out, double *result, pauli_stream_t st) {
    return guarded([&] {
        check_sum(H);
        check_sector(s);
        check_dtype(dtype);
        PS_CHECK(H->n == s->v.n, PAULI_EINVAL, "operator and sector have different qubit counts");
        check_state_ptr(psi, dtype, "psi");
        PS_CHECK(n_rows >= 0 && n_rows < (1ll << 31), PAULI_EINVAL, "n_rows must be in 0..2^31-1");
        PS_CHECK(n_rows == 0 || rows != nullptr, PAULI_EINVAL, "rows is NULL");
        PS_CHECK(hpsi_out != nullptr || result != nullptr, PAULI_EINVAL, "neither hpsi_out nor result is given");
        if (hpsi_out) {
            check_state_ptr(hpsi_out, dtype, "hpsi_out");
            const size_t bytes = (size_t)s->v.dim * elem_size(dtype);
            const char *a = static_cast<const char *>(psi);
            const char *b = static_cast<const char *>(hpsi_out);
            PS_CHECK(a + bytes <= b || b + bytes <= a, PAULI_EINVAL, "psi and hpsi_out overlap");
        }
        cudaStream_t cs = (cudaStream_t)st;
        if (n_rows == 0) {
            if (result) PS_CUDA(cudaMemsetAsync(result, 0, 4 * sizeof(double), cs));
            return;
        }
        if (result && H->rows_cap < n_rows) {
            PS_CUDA(cudaStreamSynchronize(cs));
            dev_free(H->al, H->rows_part);
            H->rows_part = nullptr;
            H->rows_cap = 0;
            H->rows_part = static_cast<double *>(dev_alloc(H->al, (size_t)n_rows * 4 * sizeof(double)));
            H->rows_cap = n_rows;
        }
        launch_apply_rows(H, s->v, psi, rows, n_rows, hpsi_out, dtype, result ? H->rows_part : nullptr, cs);
        if (result) launch_reduce(H->rows_part, n_rows, result, cs);
    });
}

int pauli_rotate(pauli_sum *G, const pauli_sector *s, double theta, void *psi, int dtype, pauli_stream_t st) {
    return guarded([&] {
        check_sum(G);
        check_sector(s);
        check_dtype(dtype);
        PS_CHECK(G->n == s->v.n, PAULI_EINVAL, "generator and sector have different qubit counts");
        PS_CHECK(std::isfinite(theta), PAULI_EINVAL, "theta must be finite");
        check_state_ptr(psi, dtype, "psi");
        if (G->m == 0) return;
        PS_CHECK(G->G == 1, PAULI_EINVAL, "rotation generator must have exactly one X mask");
        PS_CHECK(G->hermitian, PAULI_ENOTHERMITIAN, "rotation generator is not Hermitian");
        launch_rotate(G, s, theta, psi, dtype, (cudaStream_t)st);
    });
}

int pauli_rotate_adjoint(pauli_sum *G, const pauli_sector *s, double theta, void *phi, void *lam, int dtype,
                         double *result, pauli_stream_t st) {
    return guarded([&] {
        check_sum(G);
        check_sector(s);
        check_dtype(dtype);
        PS_CHECK(G->n == s->v.n, PAULI_EINVAL, "generator and sector have different qubit counts");
        PS_CHECK(std::isfinite(theta), PAULI_EINVAL, "theta must be finite");
        check_state_ptr(phi, dtype, "phi");
        check_state_ptr(lam, dtype, "lam");
        PS_CHECK(phi != lam, PAULI_EINVAL, "phi and lam must be different vectors");
        PS_CHECK(result != nullptr, PAULI_EINVAL, "result is NULL");
        PS_CHECK(G->m == 0 || G->G == 1, PAULI_EINVAL, "rotation generator must have exactly one X mask");
        PS_CHECK(G->hermitian, PAULI_ENOTHERMITIAN, "rotation generator is not Hermitian");
        if (G->m == 0) {
            PS_CUDA(cudaMemsetAsync(result, 0, 2 * sizeof(double), (cudaStream_t)st));
            return;
        }
        launch_rotate_adjoint(G, s, theta, phi, lam, dtype, result, (cudaStream_t)st);
    });
}

int pauli_status(pauli_sum *H, pauli_stream_t st, int *code) {
    return guarded([&] {
        check_sum(H);
        PS_CHECK(code != nullptr, PAULI_EINVAL, "code is NULL");
        cudaStream_t cs = (cudaStream_t)st;
        int v = 0;
        PS_CUDA(cudaMemcpyAsync(&v, H->status, sizeof(int), cudaMemcpyDeviceToHost, cs));
        PS_CUDA(cudaMemsetAsync(H->status, 0, sizeof(int), cs));
        PS_CUDA(cudaStreamSynchronize(cs));
        *code = v;
    });
}

}  // extern "C"
