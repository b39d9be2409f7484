// batch.cu -- many independent states, each with its own operator and sector,
// in persistent launches: H_b psi_b and <psi_b|H_b|psi_b> for every b.
//
// By default every state keeps the staged-gather shape a launch of its own
// would take (columns per thread, staged rows in flight, rows staged by bit
// pattern or by rank); states are grouped by shape, largest first inside a
// group, and each group is one persistent launch whose CTAs pull (state, row,
// column tile) units from an atomic counter.  A uniform shape for all states
// can be installed or found by the tuner instead.
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
    int64_t total = 0;                // work units of all launches
    bool grouped = true;              // per-state shapes (one launch per shape group)
    int tpt = 0, nbuf = 1;            // the uniform shape (grouped == false)
    bool ranked = false;              // rows staged by rank (wide splits)
    struct Group {
        int tpt, nbuf;
        bool ranked;
        int q0, q1;                   // queue positions of the group's states
        int64_t total;                // work units of the group's launch
        int max_nlo;
        int64_t max_dlo;
    };
    std::vector<Group> groups;
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
void launch_group_t(pauli_batch *b, const pauli_batch::Group &g, size_t smem, bool want_out, cudaStream_t st) {
    auto kern = k_apply_batch<R, KIND, REALH, TPT, NBUF>;
    smem_optin(reinterpret_cast<const void *>(kern), smem);
    int per_sm = 0;
    PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    const int sms = num_sms();
    PS_CHECK(per_sm >= 1, PAULI_EUNSUPPORTED, "batched apply: the launch shape does not fit on an SM");
    if (g.total <= 0) return;
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, g.total);
    PS_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st));
    kern<<<(unsigned)grid, kThreads, smem, st>>>(b->d_desc + g.q0, b->d_ptrs + g.q0, g.q1 - g.q0, g.total,
                                                 b->d_counter, b->d_partials, want_out ? 1 : 0);
    PS_LAUNCH_CHECK();
}

// Dynamic shared memory of a group's launch: its widest state decides.
size_t group_smem(const pauli_batch *b, int nbuf, bool ranked, int max_nlo, int64_t max_dlo) {
    auto bb = [&](int cap) {
        return b->dtype == PAULI_C64 ? Smem<float>::buf_bytes(cap) : Smem<double>::buf_bytes(cap);
    };
    if (!ranked) return (size_t)nbuf * bb(1 << max_nlo);
    return (size_t)nbuf * bb(ranked_rowcap(max_dlo)) + rank_table_bytes(max_nlo);
}
size_t batch_smem(const pauli_batch *b, int nbuf, bool ranked) {
    return group_smem(b, nbuf, ranked, b->max_nlo, b->max_dlo);
}

template <typename R, int KIND, bool REALH>
void launch_group_k(pauli_batch *b, const pauli_batch::Group &g, bool want_out, cudaStream_t st) {
    const size_t smem = group_smem(b, g.nbuf, KIND == KBLKR, g.max_nlo, g.max_dlo);
    PS_CHECK(smem <= 226 * 1024, PAULI_EUNSUPPORTED, "batched apply: the widest sector split is too wide");
#define PS_B(T, N) launch_group_t<R, KIND, REALH, T, N>(b, g, smem, want_out, st)
    if (g.nbuf == 2) {
        if (g.tpt == 4) PS_B(4, 2); else if (g.tpt == 2) PS_B(2, 2); else PS_B(1, 2);
    } else {
        if (g.tpt == 4) PS_B(4, 1); else if (g.tpt == 2) PS_B(2, 1); else PS_B(1, 1);
    }
#undef PS_B
}

template <typename R>
void launch_group_r(pauli_batch *b, const pauli_batch::Group &g, bool want_out, cudaStream_t st) {
    if (g.ranked) {
        if (b->realh) launch_group_k<R, KBLKR, true>(b, g, want_out, st);
        else launch_group_k<R, KBLKR, false>(b, g, want_out, st);
    } else {
        if (b->realh) launch_group_k<R, KBLK1, true>(b, g, want_out, st);
        else launch_group_k<R, KBLK1, false>(b, g, want_out, st);
    }
}

// every group's launch, then the fixed-order reduction of every state's partials
void launch_batch(pauli_batch *b, double *results, bool want_out, cudaStream_t st) {
    for (const auto &g : b->groups) {
        if (b->dtype == PAULI_C64) launch_group_r<float>(b, g, want_out, st);
        else launch_group_r<double>(b, g, want_out, st);
    }
    k_batch_reduce<<<b->n, 256, 0, st>>>(b->d_desc, b->d_partials, results);
    PS_LAUNCH_CHECK();
}

// The staged-gather shape a launch of its own would give state i (its tuned or
// heuristic shape; a list / direct / SVD choice is replaced by the staged one).
void state_shape(pauli_batch *b, int i, int &tpt, int &nbuf, bool &ranked) {
    const SectorView &v = b->S[i]->v;
    Plan *p = find_plan(b->H[i], v);
    PS_CHECK(p != nullptr, PAULI_EINVAL, "batched apply: a plan is missing (internal)");
    ApplyCfg c = apply_config(*p, v, b->dtype, false);
    if (c.list || c.direct || c.svd || c.local) {
        LaunchChoice f;
        f.direct = 0;
        c = apply_config(*p, v, b->dtype, false, &f);
    }
    tpt = c.tpt >= 4 ? 4 : c.tpt;  // the batched kernel has 1, 2 or 4 columns per thread
    nbuf = c.nbuf;
    ranked = c.ranked;
    // a pattern-staged row wider than 64 KB leaves one CTA per SM in a persistent
    // launch (a single launch hides that behind its row split): stage by rank instead
    const size_t es = b->dtype == PAULI_C64 ? 8 : 16;
    if (!ranked && (es << v.n_lo) * (size_t)nbuf > 64 * 1024 && v.n_lo <= (v.irr ? 14 : 16)) {
        ranked = true;
        tpt = 4;
        nbuf = 1;
    }
}

// (Re)build the queue: shape groups (per state, or one uniform shape), states
// largest first inside a group, descriptors and partial slots.
void build_descs(pauli_batch *b) {
    struct St {
        int i, tpt, nbuf;
        bool ranked;
        int64_t nwork;
    };
    std::vector<St> st(b->n);
    for (int i = 0; i < b->n; ++i) {
        St &e = st[i];
        e.i = i;
        if (b->grouped) {
            state_shape(b, i, e.tpt, e.nbuf, e.ranked);
        } else {
            e.tpt = b->tpt;
            e.nbuf = b->nbuf;
            e.ranked = b->ranked;
        }
        const SectorView &v = b->S[i]->v;
        // a point-group block is found by its (popcount, irrep) class, which only
        // the rank-staged kernel evaluates
        if (v.irr) e.ranked = true;
        e.nwork = make_geom(v, e.tpt * kThreads).cta_off[v.nblk];
    }
    std::stable_sort(st.begin(), st.end(), [](const St &a, const St &c) {
        if (a.ranked != c.ranked) return a.ranked < c.ranked;
        if (a.tpt != c.tpt) return a.tpt > c.tpt;
        if (a.nbuf != c.nbuf) return a.nbuf < c.nbuf;
        return a.nwork > c.nwork;
    });
    std::vector<BatchDesc> h(b->n);
    b->order.resize(b->n);
    b->groups.clear();
    int64_t part = 0;
    for (int q = 0; q < b->n; ++q) {
        const St &e = st[q];
        if (b->groups.empty() || b->groups.back().tpt != e.tpt || b->groups.back().nbuf != e.nbuf ||
            b->groups.back().ranked != e.ranked)
            b->groups.push_back({e.tpt, e.nbuf, e.ranked, q, q, 0, 0, 0});
        pauli_batch::Group &g = b->groups.back();
        const int i = e.i;
        const SectorView &v = b->S[i]->v;
        Plan *p = find_plan(b->H[i], v);
        PS_CHECK(p != nullptr, PAULI_EINVAL, "batched apply: a plan is missing (internal)");
        BatchDesc d;
        d.v = v;
        d.geo = make_geom(v, e.tpt * kThreads, 1, nullptr, (int32_t)p->P);
        d.p = plan_dev(*p);
        d.work0 = g.total;   // relative to the group's launch
        d.nwork = e.nwork;
        d.part0 = part;      // global partial slots
        h[q] = d;
        b->order[q] = i;
        g.q1 = q + 1;
        g.total += e.nwork;
        g.max_nlo = std::max(g.max_nlo, v.n_lo);
        g.max_dlo = std::max<int64_t>(g.max_dlo, v.dlo[0]);
        part += e.nwork;
    }
    b->total = part;
    dev_free(b->al, b->d_partials);
    b->d_partials = nullptr;
    b->d_partials = static_cast<double *>(dev_alloc(b->al, (size_t)std::max<int64_t>(1, part) * 4 * sizeof(double)));
    PS_CUDA(cudaMemcpy(b->d_desc, h.data(), sizeof(BatchDesc) * b->n, cudaMemcpyHostToDevice));
    PS_CUDA(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
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
                PS_CHECK(!S[i]->v.irr || S[i]->v.n_lo <= 14, PAULI_EUNSUPPORTED,
                         "batch: a point-group sector's low half must be at most 14 qubits (rank tables)");
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
            // one uniform shape by default: four columns a thread, rows staged by
            // rank (the fastest of the shapes measured on 64 molecules of 8-14
            // orbitals; per-state shape groups are an installable alternative)
            b->grouped = false;
            b->tpt = 4;
            b->nbuf = 1;
            b->ranked = true;
            build_descs(b);
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
        launch_batch(b, b->d_results, psi_out != nullptr, cs);
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
        bool bg = b->grouped;
        int bt = b->tpt, bn = b->nbuf;
        bool br = b->ranked;
        // candidates: the per-state shapes, and every uniform shape that fits
        struct Cand {
            bool grouped;
            int tpt, nbuf;
            bool ranked;
        };
        std::vector<Cand> cands{{true, 4, 1, false}};
        for (int tpt : {1, 2, 4})
            for (int ranked : {0, 1})
                for (int nbuf : {1, 2})
                    if (batch_smem(b, nbuf, ranked != 0) <= 226 * 1024) cands.push_back({false, tpt, nbuf, ranked != 0});
        try {
            for (const Cand &c : cands) {
                b->grouped = c.grouped;
                b->tpt = c.tpt;
                b->nbuf = c.nbuf;
                b->ranked = c.ranked;
                build_descs(b);
                upload_ptrs(b, psi_in, psi_out, cs);
                launch_batch(b, b->d_results, psi_out != nullptr, cs);
                PS_CUDA(cudaEventRecord(e0, cs));
                for (int r = 0; r < reps; ++r) launch_batch(b, b->d_results, psi_out != nullptr, cs);
                PS_CUDA(cudaEventRecord(e1, cs));
                PS_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                PS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms / reps < best_ms) {
                    best_ms = ms / reps;
                    bg = c.grouped;
                    bt = c.tpt;
                    bn = c.nbuf;
                    br = c.ranked;
                }
            }
        } catch (...) {
            (void)cudaEventDestroy(e0);
            (void)cudaEventDestroy(e1);
            throw;
        }
        (void)cudaEventDestroy(e0);
        (void)cudaEventDestroy(e1);
        b->grouped = bg;
        b->tpt = bt;
        b->nbuf = bn;
        b->ranked = br;
        build_descs(b);
        if (best) {
            best->cols_per_thread = bg ? 0 : bt;
            best->staged_rows = bg ? 0 : bn;
            best->row_split = 1;
            best->direct = 0;
            best->ranked = bg ? 0 : (br ? 1 : 0);
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
        if (cfg->cols_per_thread == 0) {  // back to per-state shapes
            b->grouped = true;
            build_descs(b);
            return PAULI_OK;
        }
        PS_CHECK(cfg->cols_per_thread == 1 || cfg->cols_per_thread == 2 || cfg->cols_per_thread == 4, PAULI_EINVAL,
                 "batch: cols_per_thread must be 0 (per-state shapes), 1, 2 or 4");
        PS_CHECK(cfg->staged_rows == 1 || cfg->staged_rows == 2, PAULI_EINVAL, "staged_rows must be 1 or 2");
        PS_CHECK(cfg->ranked == 0 || cfg->ranked == 1, PAULI_EINVAL, "ranked must be 0 or 1");
        PS_CHECK(cfg->row_split == 1 && cfg->direct == 0, PAULI_EUNSUPPORTED,
                 "batch: only the staged gather without row splits runs in the batched launch");
        PS_CHECK(batch_smem(b, cfg->staged_rows, cfg->ranked != 0) <= 226 * 1024, PAULI_EUNSUPPORTED,
                 "batch: this staging layout does not fit in shared memory for the widest state");
        b->grouped = false;
        b->tpt = cfg->cols_per_thread;
        b->nbuf = cfg->staged_rows;
        b->ranked = cfg->ranked != 0;
        build_descs(b);
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
    cfg->cols_per_thread = b->grouped ? 0 : b->tpt;
    cfg->staged_rows = b->grouped ? 0 : b->nbuf;
    cfg->row_split = 1;
    cfg->direct = 0;
    cfg->ranked = b->grouped ? 0 : (b->ranked ? 1 : 0);
    cfg->ms = (double)b->groups.size();  // launches per apply
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
