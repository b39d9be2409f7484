// ps_internal.cuh -- shared internals of the paulisim CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include "../../include/paulisim.h"

namespace ps {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
void clear_error();

struct Error {
    int code;
    std::string msg;
};

#define PS_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::ps::Error{PAULI_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define PS_CHECK(cond, code, msg)                          \
    do {                                                   \
        if (!(cond)) throw ::ps::Error{(code), (msg)};     \
    } while (0)

#define PS_LAUNCH_CHECK() PS_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// device memory (allocator hook)
// ---------------------------------------------------------------------------
struct Allocator {
    void *(*alloc_fn)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
Allocator current_allocator();
void set_current_allocator(const Allocator &a);

void *dev_alloc(const Allocator &a, size_t bytes);
void dev_free(const Allocator &a, void *p);

// Opts kernel `func` in to `bytes` of dynamic shared memory on the current
// device.  The attribute is per device, so the set of (device, kernel) pairs
// already raised to at least `bytes` is remembered per device (api.cu).
void smem_optin(const void *func, size_t bytes);
// SM count of the current device (cached per device ordinal).
int num_sms();

// RAII device buffer (library-internal temporaries at build time).
template <typename T>
struct DevBuf {
    Allocator al;
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const Allocator &a, size_t count) : al(a), n(count) {
        p = static_cast<T *>(dev_alloc(al, (count ? count : 1) * sizeof(T)));
    }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : al(o.al), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) { reset(); al = o.al; p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { reset(); }
    void reset() { if (p) dev_free(al, p); p = nullptr; n = 0; }
    T *release() { T *q = p; p = nullptr; n = 0; return q; }
};

// ---------------------------------------------------------------------------
// sector
// ---------------------------------------------------------------------------
constexpr int kMaxBlocks = 33;
constexpr int kMaxHalf = 24;  // largest half width with rank / unrank tables
constexpr int kMaxCls = (kMaxHalf + 1) * 8;  // half-string classes (see SectorView)

// Everything a kernel needs to know about a sector, passed by value.
//
// The class of a half string (its low or high half of the qubits) is its
// popcount, or, in a sector with point-group labels (irr = 1), popcount * 8 +
// irrep, the irrep being the XOR of the labels (0..7) of its occupied qubits:
// bit j of it is the parity of popcount(s & irr_lo[j]) (irr_hi[j] for the high
// half).  A block r is the product of the low strings of class klo[r] and the
// high strings of class khi[r]; the khi of the blocks are distinct.  Inside a
// class the strings are ranked in ascending numeric order (colex rank for
// popcount classes).
struct SectorView {
    int n, n_lo, n_hi, kind, nblk;
    int irr;                          // 1: classes carry a point-group irrep
    uint32_t irr_lo[3], irr_hi[3];    // irrep-bit masks of the two halves
    int64_t dim;
    int64_t nrows;                    // sum over blocks of D_hi
    int klo[kMaxBlocks], khi[kMaxBlocks];  // class of each block's low / high half
    int64_t off[kMaxBlocks + 1];      // first index of each block
    int64_t dlo[kMaxBlocks], dhi[kMaxBlocks];
    int64_t row_off[kMaxBlocks + 1];  // first row of each block
    int64_t lst_lo_off[kMaxBlocks];   // first entry of each block's low class in list_lo
    int64_t lst_hi_off[kMaxBlocks];   // ... and of its high class in list_hi
    const uint32_t *rank_lo;          // [2^n_lo] rank inside the string's class
    const uint32_t *rank_hi;          // [2^n_hi]
    const uint32_t *list_lo;          // [2^n_lo] strings ordered by (class, value)
    const uint32_t *list_hi;          // [2^n_hi]
    int8_t blk_of_khi[kMaxCls];       // class of the high half -> block or -1
    // (a kernel argument: kept to about 2 KB, every field read from the
    //  constant bank by every CTA)
};

__host__ __device__ __forceinline__ int ps_popc32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

// class of a low / high half string (popcount, or popcount * 8 + irrep)
__host__ __device__ __forceinline__ int half_cls(uint32_t s, int irr, const uint32_t *m) {
    int c = ps_popc32(s);
    if (irr)
        c = (c << 3) | (ps_popc32(s & m[0]) & 1) | ((ps_popc32(s & m[1]) & 1) << 1) |
            ((ps_popc32(s & m[2]) & 1) << 2);
    return c;
}
__host__ __device__ __forceinline__ int cls_lo(const SectorView &v, uint32_t s) { return half_cls(s, v.irr, v.irr_lo); }
__host__ __device__ __forceinline__ int cls_hi(const SectorView &v, uint32_t s) { return half_cls(s, v.irr, v.irr_hi); }

// ---------------------------------------------------------------------------
// apply plan: the canonical sum re-laid out for one sector split (rows = high
// n - n_lo qubits, columns = low n_lo qubits)
// ---------------------------------------------------------------------------
// A launch shape chosen by the autotuner (0 / -1: decide automatically).
struct LaunchChoice {
    int tpt = 0;      // columns per thread: 1, 2 or 4
    int nbuf = 0;     // staged source rows in flight: 1 or 2
    int nsplit = 0;   // piece ranges per row: 1..16
    int direct = -1;  // 1: direct gather (small plans), 0: staged, 2: local passes (full space),
                      // 3: per-item lists of valid pairs (single block, n_lo <= kListMaxLo),
                      // 4: SVD-factorised phases (single block, real operator; svd.cu)
    int ranked = -1;  // 1: rows staged by rank + rank table, 0: by bit pattern
};
struct TunedEntry {
    int64_t dim;
    int nblk;
    int dtype;
    LaunchChoice choice;
    double ms;
};

// Layout (all device arrays):
//   piece p   : consecutive groups sharing x_hi (so one source row per CTA row),
//               at most kItemsPerPiece items and kSegsPerPiece segments
//   item i    : one group, or a slice of a group's segments
//   segment s : terms of one group with equal z_lo, sorted by (z_lo, z_hi)
struct LocalPlan;  // local.cu
struct SvdPlan;    // svd.cu

// Lists of the valid (target, source) pairs of each distinct x_lo of a plan's
// items in one single-block sector (low half of k_lo particles, n_lo <=
// kListMaxLo, D_lo <= kListMaxDlo).  Entry of list l: the pairs of targets t_lo
// with t_lo ^ x_lo in the block, ascending in the target's rank, each packed as
// rank(t_lo) | rank(t_lo ^ x_lo) << 10 | t_lo << 20.
struct ListTab {
    int klo = -1;
    int64_t n_list = 0, n_ent = 0;
    uint32_t *ent = nullptr;     // [n_ent]
    int32_t *off = nullptr;      // [n_list + 1]
    int32_t *it_list = nullptr;  // [I] list of each item
    std::vector<int64_t> h_pc_cumw;  // [P+1] cumulative per-piece work of the list gather
};
constexpr int kListMaxLo = 12;
constexpr int64_t kListMaxDlo = 1024;
constexpr int kListCache = 2;

struct Plan {
    int n_lo = -1;
    bool merged = false;               // low Z masks merged for single-block sectors (build.cu)
    int64_t G = 0, S = 0, M = 0;      // groups, segments, terms
    int64_t P = 0, I = 0;             // pieces, items
    int32_t nseg_diag = 0;            // segments [0, nseg_diag) belong to the x = 0 group
    bool real = true;                  // every C_k real
    uint32_t *pc_xhi = nullptr;        // [P]
    int32_t *pc_i0 = nullptr;          // [P+1] item range
    uint8_t *pc_lofree = nullptr;      // [P] 1: every item has x_lo = 0 and none is of the x = 0 group
    uint32_t *it_xlo = nullptr;        // [I]
    uint32_t *it_xhi = nullptr;        // [I] x_hi of the item's group
    int32_t *it_s0 = nullptr;          // [I+1] segment range
    uint32_t *s_zlo = nullptr;         // [S]
    uint32_t *s_xhi = nullptr;         // [S] x_hi of the segment's group
    int32_t *s_t0 = nullptr;           // [S+1] term range
    uint32_t *t_zhi = nullptr;         // [M] (segment order)
    double2 *t_c64 = nullptr;          // [M] FP64 coefficients
    float2 *t_c32 = nullptr;           // [M] FP32 coefficients
    // x = 0 group, n_lo <= kDiagTabBits: the part of its terms with z_hi = 0
    // tabulated over the low bits, T(t_lo) = sum c_k (-1)^popc(z_lo,k & t_lo)
    // (FP64, and FP32 hi + lo), and the segments that keep a term with z_hi != 0
    double2 *diag_tab64 = nullptr;     // [2^n_lo]
    float2 *diag_tab32 = nullptr;      // [2 * 2^n_lo]: hi parts, then lo parts
    int32_t *diag_rest = nullptr;      // [n_diag_rest] segment indices
    int32_t n_diag_rest = 0;
    std::vector<int64_t> h_pc_cumw;   // [P+1] cumulative per-piece work estimate
    std::vector<TunedEntry> tuned;     // autotuned launch shapes per (sector, dtype)
    // reduction scratch for pauli_expect
    double *partials = nullptr;
    int64_t partials_cap = 0;
    // partial vectors of split launches (bytes)
    void *split_buf = nullptr;
    int64_t split_cap = 0;
    // complex128 list gather: psi split into hi / lo FP32 pairs (dim elements)
    float4 *df_buf = nullptr;
    int64_t df_cap = 0;
    // SVD-factorised phases (built when that gather is installed or tuned)
    SvdPlan *svd = nullptr;
    // full-space passes over local bit sets (built on first use with a full sector)
    LocalPlan *local = nullptr;
    LocalPlan *local_cl = nullptr;   // the same with windows shared by CTA clusters
    bool local_tried = false;
    // host copies of the item tables (list building)
    std::vector<uint32_t> h_it_xlo;
    std::vector<int32_t> h_it_s0, h_pc_i0;
    ListTab lists[kListCache];   // per k_lo of the single-block sectors seen
    int nlists = 0;
};

constexpr int kDiagTabBits = 12;

// Full-space apply in passes over local bit sets (local.cu): 2^kLocBits amplitudes
// per chunk, the kLocRun lowest bits always local (runs of 8 contiguous amplitudes).
constexpr int kLocBits = 13;
constexpr int kLocRun = 3;
constexpr int kLocClusterBits = 3;  // clustered windows: 8 CTAs, kLocBits + 3 bits
constexpr int kLocMaxPass = 4;
constexpr int kLocMaxTerms = 2048;
constexpr int kLocMaxGroups = 512;

// Pairs {t, t ^ x} of a single-group rotation on a single-block sector with both
// members in the block, each listed once (the member with the lowest bit of x
// set): pair i = h * nlo + l has t = (pat_hi[h] << n_lo) | pat_lo[l], index of t
// off + rt_hi[h] * D_lo + rt_lo[l] and index of t ^ x off + rs_hi[h] * D_lo + rs_lo[l].
// Active pair patterns of a single-X-mask sum G = sum_k C_k X^x Z^{z_k}.
// With D = OR_k (z_k ^ z_0), S = x | D and z_o = z_0 & ~S,
//   f(s) = sum_k C_k (-1)^{z_k . s} = (-1)^{z_o . s} F(s & S),
// so whether a pair {t, t ^ x} rotates, and by how much, depends only on the
// pattern q = t & S.  np > 0: the np patterns q (bit b0 of x set; any q when
// x = 0) with F(q ^ x) != 0 and those F values, summed in the order of the
// terms; np = -1: no pattern is active; np = 0: not tabulated (S wider than
// 14 bits or more than kActMax active patterns).
constexpr int kActMax = 4;
struct ActivePatterns {
    uint64_t S = 0, zo = 0;
    uint64_t pat[kActMax] = {};
    double2 F[kActMax] = {};
    int np = 0;
};
ActivePatterns find_active_patterns(uint64_t x, const uint64_t *z, const double2 *c, int64_t m);  // rotseq.cu

struct RotPairs {
    uint64_t sector_uid = 0;
    int leaks = -1;            // the generator moves amplitude out of the sector: -1 unknown
    int64_t nlo = 0, nhi = 0;  // table entries per half
    uint32_t *tab = nullptr;   // pat_lo, rt_lo, rs_lo [nlo] each, then pat_hi, rt_hi, rs_hi [nhi]
    ActivePatterns act;        // the generator's active patterns (np > 0: angles per pattern on the host)
};
constexpr int kRotPairsCache = 4;
constexpr int kRotPairTerms = 512;  // generators with more terms keep the per-target kernel

struct PlanLimits {
    static constexpr int kItemsPerPiece = 64;
    static constexpr int kSegsPerPiece = 512;
};

}  // namespace ps

// ---------------------------------------------------------------------------
// opaque handles
// ---------------------------------------------------------------------------
struct pauli_sum {
    uint32_t magic;
    ps::Allocator al;
    int n;
    int64_t m = 0, G = 0;
    bool real = true;        // every C imaginary part == 0
    bool hermitian = true;   // letter-form coefficients real (within 1e-12 max|C|)
    double cmax = 0.0;
    uint64_t *x = nullptr, *z = nullptr;  // [m] canonical
    double2 *c = nullptr;                 // [m]
    uint64_t *gx = nullptr;               // [G]
    int64_t *gstart = nullptr;            // [G+1]
    int *status = nullptr;                // device status word
    uint64_t gx0_host = 0;                // gx[0] read back once (single-group rotations)
    bool gx0_known = false;
    ps::RotPairs rot[ps::kRotPairsCache];   // pair tables per sector (single-group rotations)
    int nrot = 0;
    int *leak_flag = nullptr;             // device word of the one-time leak check
    ps::Plan plans[4];
    int nplans = 0;
    double *rows_part = nullptr;          // [rows_cap][4] partials of pauli_expect_rows
    int64_t rows_cap = 0;
};

struct pauli_sector {
    uint32_t magic;
    ps::Allocator al;
    uint64_t uid = 0;  // unique per created sector (keys caches held by operators)
    ps::SectorView v;
    uint32_t *tables = nullptr;  // backing store of rank / list tables
};

namespace ps {
constexpr uint32_t kSumMagic = 0x50534d31u;     // "PSM1"
constexpr uint32_t kSectorMagic = 0x50534331u;  // "PSC1"

// rows.cu: selected rows of H psi (one CTA per target index)
void launch_apply_rows(const pauli_sum *H, const SectorView &v, const void *psi, const int64_t *rows, int64_t nrows,
                       void *out, int dtype, double *partials, cudaStream_t st);

// build.cu
void to_xz_device(int64_t m, const uint64_t *x, const uint64_t *z, const uint8_t *gamma,
                  const double *cre, const double *cim, int letter, double2 *out, cudaStream_t st);
void canonicalize(pauli_sum *h, int64_t m, uint64_t *d_x, uint64_t *d_z, double2 *d_c,
                  double eps_drop, cudaStream_t st);
void jw_molecular_raw_device(int norb, const double *h, const double *g, double e_nn,
                             double eps_int, const Allocator &al, DevBuf<uint64_t> &x,
                             DevBuf<uint64_t> &z, DevBuf<double2> &c, int64_t &count,
                             cudaStream_t st);
void jw_fermion_raw_device(int n, int nterms, const int *nf, const int *modes, const int *dag,
                           const double *cre, const double *cim, const Allocator &al,
                           DevBuf<uint64_t> &x, DevBuf<uint64_t> &z, DevBuf<double2> &c,
                           int64_t &count, cudaStream_t st);
// Plans are keyed by (n_lo, merged): a single-block sector uses a plan whose
// segments merge the low Z masks z_lo and z_lo ^ x_lo (exact on every pair the
// sector keeps), other sectors the plain plan.
inline bool plan_merges(const SectorView &v) { return v.kind == PAULI_SECTOR_BLOCKS && v.nblk == 1; }
Plan &get_plan(pauli_sum *h, const SectorView &v, cudaStream_t st);
Plan *find_plan(pauli_sum *h, const SectorView &v);  // existing plan or nullptr; never builds
void free_plan(const Allocator &al, Plan &p);

// scan.cu
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, const Allocator &al,
                        cudaStream_t st);
// Stable LSD radix sort of (hi, lo) 128-bit keys over the given significant
// bit counts; perm receives the original index of each sorted element.
void radix_sort_keys(uint64_t *hi, uint64_t *lo, int64_t *perm, int64_t n, int hi_bits,
                     int lo_bits, const Allocator &al, cudaStream_t st);

// sector.cu
void build_sector_tables(pauli_sector *s, cudaStream_t st);
void sector_rank(const SectorView &v, const uint64_t *cfg, int64_t n, int64_t *idx, cudaStream_t st);
void sector_unrank(const SectorView &v, const int64_t *idx, int64_t n, uint64_t *cfg,
                   cudaStream_t st);

// apply.cu
struct ApplyCfg {
    int tpt = 1;            // targets (columns) per thread
    int nbuf = 1;           // staged source rows in flight (1 or 2)
    size_t smem = 0;        // dynamic shared memory per CTA
    int64_t base_nct = 0;   // (row, column tile) CTAs
    int nsplit = 1;         // piece ranges per (row, tile)
    std::vector<int32_t> split_p0;
    int64_t nct = 0;        // CTAs of the gather launch = base_nct * nsplit
    int64_t combine_nct = 0;
    bool direct = false;    // small plan: k_apply_direct (no staging, no split)
    bool local = false;     // full space: passes over local bit sets (local.cu)
    bool local_cl = false;  // ... with the windows shared by CTA clusters (reported as ranked = 1)
    bool ranked = false;    // single block, rows staged by rank (KBLKR)
    bool list = false;      // single block, n_lo <= kListMaxLo: per-item lists of valid pairs (list.cu)
    bool svd = false;       // single block, real operator: SVD-factorised phases (svd.cu)
};
ApplyCfg apply_config(const Plan &p, const SectorView &v, int dtype, bool allow_split,
                      const LaunchChoice *force = nullptr);
void launch_apply(pauli_sum *H, const Plan &p, const SectorView &v, const void *psi_in,
                  void *psi_out, int dtype, double *partials, cudaStream_t st, bool allow_split = true,
                  const LaunchChoice *force = nullptr);
void launch_reduce(const double *partials, int64_t nparts, double *result, cudaStream_t st);
// number of 4-double partial-sum slots an expectation launch writes
int64_t apply_num_ctas(const Plan &p, const SectorView &v, int dtype, bool allow_split = true,
                       const LaunchChoice *force = nullptr);
// elements of the split scratch a launch needs (0: no split)
int64_t apply_split_elems(const Plan &p, const SectorView &v, int dtype, const LaunchChoice *force = nullptr);
void launch_rotate(pauli_sum *G, const pauli_sector *s, double theta, void *psi, int dtype, cudaStream_t st);
// X mask of a single-group operator (read back once and kept in G)
uint64_t group_mask0(pauli_sum *G);
// Pair tables of a single-group generator on a single-block sector (built on
// first use, with a one-time leak check that synchronises st), or nullptr where
// the per-target kernels apply (full space, several blocks, x = 0, more than
// kRotPairTerms terms, or a generator that leaks out of the sector).
const RotPairs *rotation_pairs(pauli_sum *G, const pauli_sector *sec, uint64_t x, cudaStream_t st);
// <lam|G|phi> into result[0..1] (device), then phi, lam <- exp(-i theta G) phi, lam
void launch_rotate_adjoint(pauli_sum *G, const pauli_sector *s, double theta, void *phi, void *lam, int dtype,
                           double *result, cudaStream_t st);

// list.cu
// Builds what a sector needs beyond the plan: the local-pass plan of a full
// space, the pair lists of a single-block sector.
void prepare_for_sector(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st);
const ListTab *find_lists(const Plan &p, int klo);
void free_lists(const Allocator &al, Plan &p);
size_t list_smem(int dtype, int64_t dlo);
void launch_list(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out, int dtype,
                 double *partials, void *split_buf, cudaStream_t st);
// allocates the double-float copy of psi that the complex128 list gather reads,
// when the plan's complex128 launch shape for this sector is the list gather
void ensure_df_capacity(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st);
void ensure_df_buffer(pauli_sum *H, Plan &p, const SectorView &v, cudaStream_t st);  // unconditionally

// svd.cu
SvdPlan *build_svd_plan(pauli_sum *H, const SectorView &v, cudaStream_t st);
void free_svd_plan(SvdPlan *sp);
bool svd_plan_fits(const SvdPlan *sp, const SectorView &v);  // built for this sector's low half
size_t svd_smem(const SectorView &v, int dtype);
int svd_batches(const SvdPlan *sp);
const std::vector<int> &svd_rank_hist(const SvdPlan *sp);
void launch_svd(const ApplyCfg &cfg, const Plan &p, const SectorView &v, const void *in, void *out, int dtype,
                double *partials, cudaStream_t st);

// local.cu
LocalPlan *build_local_plan(pauli_sum *H, int n, bool cluster, cudaStream_t st);
void free_local_plan(LocalPlan *lp);
int64_t local_last_chunks(const LocalPlan *lp);
// bytes of the plan's H psi scratch (used when the caller passes no output vector)
int64_t local_scratch_bytes(const LocalPlan *lp);
int local_passes(const LocalPlan *lp);
void launch_local(LocalPlan *lp, const void *in, void *out, int dtype, int64_t dim, double *partials, int tpt,
                  cudaStream_t st);

// linalg.cu: per-device scratch of FP64 partial sums shared by the reductions
// that run on a fixed grid (pauli_vdot, pauli_rotate_adjoint)
struct DotScratch {
    double *partials = nullptr;  // [blocks][4]
    int blocks = 0;
};
DotScratch &dot_scratch();
void launch_reduce2(const double *partials, int64_t nparts, double *result, cudaStream_t st);
}  // namespace ps
