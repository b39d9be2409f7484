// batch.cu -- many independent states, each with its own operator and sector,
// in one persistent launch: H_b psi_b and <psi_b|H_b|psi_b> for every b.
#include <algorithm>
#include <cfloat>
#include <numeric>
#include <vector>

#include "apply_kernels.cuh"

using namespace ps;

struct pauli_batch {
    uint32_t magic;
    Allocator al;
    int n = 0, dtype = PAULI_C64;
    bool realh = true;
    std::vector<pauli_sum *> H;
    std::vector<const pauli_sector *> S;
    std::vector<int> order;           // queue position -> state
    std::vector<int64_t> rw_bits;     // n_lo per state
    int max_nlo = 0;
    int64_t max_dlo = 0;
    int64_t total = 0;                // work units of one launch
    int tpt = 0, nbuf = 1;            // launch shape (0: not chosen yet)
    bool ranked = false;              // rows staged by rank (wide splits)
    BatchDesc *d_desc = nullptr;      // [n] in queue order
    BatchPtrs *d_ptrs = nullptr;      // [n]
    double *d_partials = nullptr;     // [total][4]
    double *d_results = nullptr;      // [n][4] in queue order
    unsigned long long *d_counter = nullptr;
    int *d_order = nullptr;           // [n] queue position -> state
    std::vector<BatchPtrs> h_ptrs;
};

namespace ps_batch {
constexpr uint32_t kBatchMagic = 0x50424131u;

template <typename R, int KIND, bool REALH, int TPT, int NBUF>
void launch_batch_t(pauli_batch *b, size_t smem, double *results, bool want_out, cudaStream_t st) {
    auto kern = k_apply_batch<R, KIND, REALH, TPT, NBUF>;
    smem_optin(reinterpret_cast<const void *>(kern), smem);
    int per_sm = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    const int sms = num_sms();
    PS_CHECK(per_sm >= 1, PAULI_EUNSUPPORTED, "batched apply: the launch shape does not fit on an SM");
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(1, b->total));
    PS_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st));
    kern<<<(unsigned)grid, kThreads, smem, st>>>(b->d_desc, b->d_ptrs, b->n, b->total, b->d_counter, b->d_partials,
                                                 want_out ? 1 : 0);
    PS_LAUNCH_CHECK();
    k_batch_reduce<<<b->n, 256, 0, st>>>(b->d_desc, b->d_partials, results);
    PS_LAUNCH_CHECK();
}

// Dynamic shared memory of the batched launch: the widest state decides.
size_t batch_smem(const pauli_batch *b, int nbuf, bool ranked) {
    auto bb = [&](int cap) {
        return b->dtype == PAULI_C64 ? Smem<float>::buf_bytes(cap) : Smem<double>::buf_bytes(cap);
    };
    if (!ranked) return (size_t)nbuf * bb(1 << b->max_nlo);
    return (size_t)nbuf * bb(ranked_rowcap(b->max_dlo)) + rank_table_bytes(b->max_nlo);
}

template <typename R, int KIND, bool REALH>
void launch_batch_k(pauli_batch *b, int tpt, int nbuf, double *results, bool want_out, cudaStream_t st) {
    const size_t smem = batch_smem(b, nbuf, KIND == KBLKR);
    PS_CHECK(smem <= 226 * 1024, PAULI_EUNSUPPORTED, "batched apply: the widest sector split is too wide");
#define PS_B(T, N) launch_batch_t<R, KIND, REALH, T, N>(b, smem, results, want_out, st)
    if (nbuf == 2) {
        if (tpt == 4) PS_B(4, 2); else if (tpt == 2) PS_B(2, 2); else PS_B(1, 2);
    } else {
        if (tpt == 4) PS_B(4, 1); else if (tpt == 2) PS_B(2, 1); else PS_B(1, 1);
    }
#undef PS_B
}

template <typename R>
void launch_batch_r(pauli_batch *b, int tpt, int nbuf, bool ranked, double *results, bool want_out, cudaStream_t st) {
    if (ranked) {
        if (b->realh) launch_batch_k<R, KBLKR, true>(b, tpt, nbuf, results, want_out, st);
        else launch_batch_k<R, KBLKR, false>(b, tpt, nbuf, results, want_out, st);
    } else {
        if (b->realh) launch_batch_k<R, KBLK1, true>(b, tpt, nbuf, results, want_out, st);
        else launch_batch_k<R, KBLK1, false>(b, tpt, nbuf, results, want_out, st);
    }
}

void launch_batch(pauli_batch *b, int tpt, int nbuf, bool ranked, double *results, bool want_out, cudaStream_t st) {
    if (b->dtype == PAULI_C64) launch_batch_r<float>(b, tpt, nbuf, ranked, results, want_out, st);
    else launch_batch_r<double>(b, tpt, nbuf, ranked, results, want_out, st);
}

// (Re)build the descriptors for a columns-per-thread value.
void build_descs(pauli_batch *b, int tpt) {
    std::vector<BatchDesc> h(b->n);
    std::vector<int64_t> nwork(b->n);
    for (int i = 0; i < b->n; ++i) {
        const SectorView &v = b->S[i]->v;
        nwork[i] = make_geom(v, tpt * kThreads).cta_off[v.nblk];
    }
    b->order.resize(b->n);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) { return nwork[a] > nwork[c]; });
    int64_t w0 = 0;
    for (int q = 0; q < b->n; ++q) {
        const int i = b->order[q];
        const SectorView &v = b->S[i]->v;
        Plan *p = find_plan(b->H[i], v);
        PS_CHECK(p != nullptr, PAULI_EINVAL, "batched apply: a plan is missing (internal)");
        BatchDesc d;
        d.v = v;
        d.geo = make_geom(v, tpt * kThreads, 1, nullptr, (int32_t)p->P);
        d.p = plan_dev(*p);
        d.work0 = w0;
        d.nwork = nwork[i];
        d.part0 = w0;
        h[q] = d;
        w0 += nwork[i];
    }
    b->total = w0;
    dev_free(b->al, b->d_partials);
    b->d_partials = nullptr;
    b->d_partials = static_cast<double *>(dev_alloc(b->al, (size_t)std::max<int64_t>(1, w0) * 4 * sizeof(double)));
    PS_CUDA(cudaMemcpy(b->d_desc, h.data(), sizeof(BatchDesc) * b->n, cudaMemcpyHostToDevice));
    PS_CUDA(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
    b->tpt = tpt;
}

void upload_ptrs(pauli_batch *b, const void *const *psi_in, void *const *psi_out, cudaStream_t st) {
    for (int q = 0; q < b->n; ++q) {
        const int i = b->order[q];
        b->h_ptrs[q].in = psi_in[i];
        b->h_ptrs[q].out = psi_out ? psi_out[i] : nullptr;
    }
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    PS_CUDA(cudaMemcpyAsync(b->d_ptrs, b->h_ptrs.data(), sizeof(BatchPtrs) * b->n, cudaMemcpyHostToDevice, st));
}

__global__ void k_unpermute(const double *src, const int *order, int n, double *dst) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    for (int k = 0; k < 4; ++k) dst[(int64_t)order[q] * 4 + k] = src[(int64_t)q * 4 + k];
}
}  // namespace ps_batch

using namespace ps_batch;

extern "C" {

int pauli_batch_create(int n, pauli_sum *const *H, const pauli_sector *const *S, int dtype, pauli_batch **out) {
    try {
        clear_error();
        PS_CHECK(out != nullptr, PAULI_EINVAL, "out is NULL");
        *out = nullptr;
        PS_CHECK(n >= 1 && n <= 1 << 16, PAULI_EINVAL, "n must be in 1..65536");
        PS_CHECK(H && S, PAULI_EINVAL, "handle arrays are NULL");
        PS_CHECK(dtype == PAULI_C64 || dtype == PAULI_C128, PAULI_EINVAL, "bad dtype");
        pauli_batch *b = new pauli_batch();
        b->magic = kBatchMagic;
        b->al = current_allocator();
        b->n = n;
        b->dtype = dtype;
        try {
            for (int i = 0; i < n; ++i) {
                PS_CHECK(H[i] && H[i]->magic == kSumMagic, PAULI_EINVAL, "batch: invalid pauli_sum handle");
                PS_CHECK(S[i] && S[i]->magic == kSectorMagic, PAULI_EINVAL, "batch: invalid pauli_sector handle");
                PS_CHECK(H[i]->n == S[i]->v.n, PAULI_EINVAL, "batch: operator / sector qubit counts differ");
                PS_CHECK(S[i]->v.kind == PAULI_SECTOR_BLOCKS && S[i]->v.nblk == 1, PAULI_EUNSUPPORTED,
                         "batch: every sector must be a single product block (k_lo, k_hi)");
                int rc = pauli_prepare(H[i], S[i]);
                if (rc != PAULI_OK) throw Error{rc, std::string("batch: ") + pauli_last_error()};
                b->H.push_back(H[i]);
                b->S.push_back(S[i]);
                b->realh = b->realh && H[i]->real;
                b->max_nlo = std::max(b->max_nlo, S[i]->v.n_lo);
                b->max_dlo = std::max<int64_t>(b->max_dlo, S[i]->v.dlo[0]);
            }
            PS_CHECK(b->max_nlo <= 16, PAULI_EUNSUPPORTED, "batch: the low half of a split is wider than 16 qubits");
            b->d_desc = static_cast<BatchDesc *>(dev_alloc(b->al, sizeof(BatchDesc) * n));
            b->d_ptrs = static_cast<BatchPtrs *>(dev_alloc(b->al, sizeof(BatchPtrs) * n));
            b->d_results = static_cast<double *>(dev_alloc(b->al, sizeof(double) * 4 * n));
            b->d_counter = static_cast<unsigned long long *>(dev_alloc(b->al, sizeof(unsigned long long)));
            b->d_order = static_cast<int *>(dev_alloc(b->al, sizeof(int) * n));
            b->h_ptrs.resize(n);
            int64_t mx = 0;
            for (int i = 0; i < n; ++i) mx = std::max<int64_t>(mx, S[i]->v.dlo[0]);
            const int tpt = mx >= 3 * kThreads ? 4 : (mx >= 3 * kThreads / 2 ? 2 : 1);
            build_descs(b, (tpt == 1 || tpt == 2 || tpt == 4) ? tpt : 1);
            b->nbuf = 1;
            b->ranked = batch_smem(b, 1, false) > 226 * 1024;
        } catch (...) {
            dev_free(b->al, b->d_desc);
            dev_free(b->al, b->d_ptrs);
            dev_free(b->al, b->d_results);
            dev_free(b->al, b->d_counter);
            dev_free(b->al, b->d_partials);
            dev_free(b->al, b->d_order);
            delete b;
            throw;
        }
        *out = b;
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_batch_apply(pauli_batch *b, const void *const *psi_in, void *const *psi_out, double *results,
                      pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(b && b->magic == kBatchMagic, PAULI_EINVAL, "not a valid pauli_batch handle");
        PS_CHECK(psi_in != nullptr, PAULI_EINVAL, "psi_in is NULL");
        for (int i = 0; i < b->n; ++i) {
            PS_CHECK(psi_in[i] && ((uintptr_t)psi_in[i] % 16) == 0, PAULI_EINVAL, "batch: psi_in entry NULL or misaligned");
            if (psi_out && psi_out[i]) {
                PS_CHECK(((uintptr_t)psi_out[i] % 16) == 0, PAULI_EINVAL, "batch: psi_out entry misaligned");
                const size_t bytes = (size_t)b->S[i]->v.dim * (b->dtype == PAULI_C64 ? 8 : 16);
                const char *a = static_cast<const char *>(psi_in[i]);
                const char *c = static_cast<const char *>(psi_out[i]);
                PS_CHECK(a + bytes <= c || c + bytes <= a, PAULI_EINVAL, "batch: psi_in and psi_out overlap");
            }
        }
        cudaStream_t cs = (cudaStream_t)st;
        upload_ptrs(b, psi_in, psi_out, cs);
        launch_batch(b, b->tpt, b->nbuf, b->ranked, b->d_results, psi_out != nullptr, cs);
        if (results) {  // results in the caller's state order
            k_unpermute<<<(b->n + 127) / 128, 128, 0, cs>>>(b->d_results, b->d_order, b->n, results);
            PS_LAUNCH_CHECK();
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

int pauli_batch_tune(pauli_batch *b, const void *const *psi_in, void *const *psi_out, int reps,
                     pauli_launch_config *best, pauli_stream_t st) {
    try {
        clear_error();
        PS_CHECK(b && b->magic == kBatchMagic, PAULI_EINVAL, "not a valid pauli_batch handle");
        PS_CHECK(psi_in != nullptr, PAULI_EINVAL, "psi_in is NULL");
        PS_CHECK(reps >= 1 && reps <= 1000, PAULI_EINVAL, "reps must be in 1..1000");
        cudaStream_t cs = (cudaStream_t)st;
        cudaEvent_t e0, e1;
        PS_CUDA(cudaEventCreate(&e0));
        PS_CUDA(cudaEventCreate(&e1));
        double best_ms = DBL_MAX;
        int bt = b->tpt, bn = b->nbuf;
        bool br = b->ranked;
        try {
            for (int tpt : {1, 2, 4}) {
                build_descs(b, tpt);
                upload_ptrs(b, psi_in, psi_out, cs);
                for (int ranked : {0, 1})
                    for (int nbuf : {1, 2}) {
                        if (batch_smem(b, nbuf, ranked != 0) > 226 * 1024) continue;
                        launch_batch(b, tpt, nbuf, ranked != 0, b->d_results, psi_out != nullptr, cs);
                        PS_CUDA(cudaEventRecord(e0, cs));
                        for (int r = 0; r < reps; ++r)
                            launch_batch(b, tpt, nbuf, ranked != 0, b->d_results, psi_out != nullptr, cs);
                        PS_CUDA(cudaEventRecord(e1, cs));
                        PS_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        if (ms / reps < best_ms) {
                            best_ms = ms / reps;
                            bt = tpt;
                            bn = nbuf;
                            br = ranked != 0;
                        }
                    }
            }
        } catch (...) {
            (void)cudaEventDestroy(e0);
            (void)cudaEventDestroy(e1);
            throw;
        }
        (void)cudaEventDestroy(e0);
        (void)cudaEventDestroy(e1);
        build_descs(b, bt);
        b->nbuf = bn;
        b->ranked = br;
        if (best) {
            best->cols_per_thread = bt;
            best->staged_rows = bn;
            best->row_split = 1;
            best->direct = 0;
            best->ranked = br ? 1 : 0;
            best->ms = best_ms;
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

int pauli_batch_set_launch_config(pauli_batch *b, const pauli_launch_config *cfg) {
    try {
        clear_error();
        PS_CHECK(b && b->magic == kBatchMagic, PAULI_EINVAL, "not a valid pauli_batch handle");
        PS_CHECK(cfg != nullptr, PAULI_EINVAL, "cfg is NULL");
        PS_CHECK(cfg->cols_per_thread == 1 || cfg->cols_per_thread == 2 || cfg->cols_per_thread == 4, PAULI_EINVAL,
                 "batch: cols_per_thread must be 1, 2 or 4");
        PS_CHECK(cfg->staged_rows == 1 || cfg->staged_rows == 2, PAULI_EINVAL, "staged_rows must be 1 or 2");
        PS_CHECK(cfg->ranked == 0 || cfg->ranked == 1, PAULI_EINVAL, "ranked must be 0 or 1");
        PS_CHECK(cfg->row_split == 1 && cfg->direct == 0, PAULI_EUNSUPPORTED,
                 "batch: only the staged gather without row splits runs in the batched launch");
        PS_CHECK(batch_smem(b, cfg->staged_rows, cfg->ranked != 0) <= 226 * 1024, PAULI_EUNSUPPORTED,
                 "batch: this staging layout does not fit in shared memory for the widest state");
        build_descs(b, cfg->cols_per_thread);
        b->nbuf = cfg->staged_rows;
        b->ranked = cfg->ranked != 0;
        return PAULI_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (...) {
        set_error("unexpected internal error");
        return PAULI_EINVAL;
    }
}

int pauli_batch_get_launch_config(const pauli_batch *b, pauli_launch_config *cfg) {
    if (!b || b->magic != kBatchMagic || !cfg) {
        set_error("invalid pauli_batch handle or NULL cfg");
        return PAULI_EINVAL;
    }
    clear_error();
    cfg->cols_per_thread = b->tpt;
    cfg->staged_rows = b->nbuf;
    cfg->row_split = 1;
    cfg->direct = 0;
    cfg->ranked = b->ranked ? 1 : 0;
    cfg->ms = 0.0;
    return PAULI_OK;
}

int pauli_batch_destroy(pauli_batch *b) {
    if (!b) return PAULI_OK;
    if (b->magic != kBatchMagic) {
        set_error("not a valid pauli_batch handle");
        return PAULI_EINVAL;
    }
    dev_free(b->al, b->d_desc);
    dev_free(b->al, b->d_ptrs);
    dev_free(b->al, b->d_results);
    dev_free(b->al, b->d_counter);
    dev_free(b->al, b->d_partials);
    dev_free(b->al, b->d_order);
    b->magic = 0;
    delete b;
    return PAULI_OK;
}

}  // extern "C"
