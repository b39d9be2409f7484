/*
 * paulisim.h -- C ABI of the GB300 (sm_103a) Pauli-algebra operator-state library.
 *
 * The library holds Pauli-sum operators H = sum_j C_j X^{x_j} Z^{z_j} in binary
 * symplectic form (Sec. 2.2-2.3 of "A High-Performance Pauli-Algebra Framework
 * for Large-Scale Quantum Simulations"), canonically reduced and grouped by
 * their X masks (eq. topological_group), and applies them to state vectors
 * with a target-driven gather (eq. reverse_sum) over spin-resolved product
 * sectors (eq. sreverse_sum, eq. fcidim).  Every step runs in the library's
 * own CUDA kernels on one GPU.
 *
 * Conventions
 *   - Qubit k is bit k of a basis configuration b (qubit 0 = least significant
 *     bit, eq. xp_encoding / zp_encoding), n_qubits <= 64.
 *   - X^x Z^z |b> = (-1)^popcount(z & b) |b XOR x>.
 *   - A term's coefficient is stored in XZ form: C = c * i^(gamma + popcount(x & z))
 *     for a LETTER-form input c (where a qubit with both bits set is the letter
 *     Y), or C = c * i^gamma for an XZ-form input (Sec. 2.2.2, Lambda = i^chi).
 *   - Canonical form (Sec. 2.3): unique (x, z) sorted ascending as unsigned
 *     (x first, then z), each coefficient the left-to-right sum of its input
 *     entries in input order, terms with re*re + im*im <= eps_drop^2 dropped.
 *   - A sector is the full 2^n space (index = configuration) or a union of
 *     product blocks r = (k_lo, k_hi): the low n_lo qubits hold k_lo ones and
 *     the high n - n_lo qubits hold k_hi ones (for a molecule in blocked spin
 *     order, alpha = low qubits, beta = high qubits, n_lo = n_orb).  Block
 *     indices follow the order given; inside block r
 *         index = off_r + rank(b_hi) * D_lo^r + rank(b_lo),
 *     rank = colex rank among strings of the same popcount (= ascending
 *     numeric order), D_lo^r = C(n_lo, k_lo).  The k_hi of the blocks must be
 *     distinct.
 *   - State vectors are caller-owned DEVICE arrays of interleaved complex
 *     numbers: PAULI_C64 = (float re, float im), PAULI_C128 = (double re,
 *     double im), indexed by sector index, 16-byte aligned.
 *   - Work is enqueued on the caller's CUDA stream (`pauli_stream_t` is a
 *     cudaStream_t; NULL = legacy default stream).  Calls return once the work
 *     is enqueued unless stated otherwise.
 *   - Every call returns PAULI_OK (0) or a negative status; the message of the
 *     last failure on the calling thread is pauli_last_error().  The library
 *     never aborts or exits.  Errors detected on the device (a rotation that
 *     leaves the sector) are recorded in a per-handle status word read by
 *     pauli_status().
 *   - Ownership: handles own their device tables and are released by the
 *     matching *_destroy call.  The library never frees caller memory.
 */
#ifndef PAULISIM_H
#define PAULISIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pauli_status_code {
    PAULI_OK = 0,
    PAULI_EINVAL = -1,          /* bad argument (null pointer, size, alias, range)  */
    PAULI_ENOMEM = -2,          /* device or host allocation failed                 */
    PAULI_ECUDA = -3,           /* a CUDA runtime call failed                        */
    PAULI_ESECTOR = -4,         /* a rotation would take amplitude out of the sector */
    PAULI_ENOTHERMITIAN = -5,   /* rotation generator is not Hermitian               */
    PAULI_ETIMEOUT = -6,        /* a bounded device wait gave up                     */
    PAULI_EUNSUPPORTED = -7     /* valid request outside what this build supports    */
};

enum pauli_dtype { PAULI_C64 = 0, PAULI_C128 = 1 };
enum pauli_coeff_form { PAULI_LETTER = 0, PAULI_XZ = 1 };
enum pauli_sector_kind { PAULI_SECTOR_FULL = 0, PAULI_SECTOR_BLOCKS = 1 };

typedef struct pauli_sum pauli_sum;
typedef struct pauli_sector pauli_sector;
typedef void *pauli_stream_t;

/* ------------------------------------------------------------------------- */
/* library                                                                    */
/* ------------------------------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next library call on the same thread. */
const char *pauli_last_error(void);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int pauli_version(void);

/* Device allocator for handle tables and plans (default: cudaMalloc/cudaFree).
 * alloc_fn(bytes, ctx) returns a device pointer or NULL; free_fn(ptr, ctx).
 * Passing NULL for both restores the default.  Handles remember the allocator
 * they were created with. */
int pauli_set_allocator(void *(*alloc_fn)(size_t bytes, void *ctx),
                        void (*free_fn)(void *ptr, void *ctx), void *ctx);

/* ------------------------------------------------------------------------- */
/* Pauli sums (Sec. 2.3: binary symplectic arrays X, Z, C; canonical form)    */
/* ------------------------------------------------------------------------- */

/* Canonical reduction of m input terms (host arrays): sort by (x, z) with a
 * stable radix sort, sum duplicates in input order, drop |C| <= eps_drop,
 * then group by x (eq. topological_group).  gamma may be NULL (all 0);
 * coeff_form is PAULI_LETTER or PAULI_XZ.  Masks must not have bits at or
 * above n_qubits (PAULI_EINVAL).  Blocking: returns when the handle is ready. */
int pauli_sum_build(int n_qubits, int64_t m, const uint64_t *x, const uint64_t *z,
                    const uint8_t *gamma, const double *c_re, const double *c_im, int coeff_form,
                    double eps_drop, pauli_sum **out);

/* Jordan-Wigner qubit Hamiltonian of Algorithm 1 for n_orb spatial orbitals
 * (2 n_orb qubits, blocked spin order: spin orbital p-alpha = qubit p,
 * p-beta = qubit n_orb + p) from host integrals h[n_orb^2] (row-major h_pq)
 * and g[n_orb^4] (chemist (pq|rs), row-major):
 *   H = sum_{s,pq} h_pq a+_{ps} a_{qs}
 *     + 1/2 sum_{s,t,pqrs} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs} + e_nn,
 * a_P = 1/2 (X_P + i Y_P) Z_{<P}.  Integrals with |v| <= eps_int are skipped,
 * as are two-body terms with P == R or Q == S (identically zero).  Raw entry
 * order: the e_nn identity entry (if e_nn != 0), one-body (s, p, q ascending,
 * 4 entries each), two-body (s, t, p, q, r, s ascending, 16 each), entries of
 * one term in expansion order with the left factor most significant; then
 * canonical reduction with eps_drop.  n_orb <= 32.  Blocking. */
int pauli_jw_molecular(int n_orb, const double *h, const double *g, double e_nn, double eps_int,
                       double eps_drop, pauli_sum **out);

/* The raw (pre-reduction) entries of pauli_jw_molecular in XZ form, written to
 * host arrays of *count entries; with x == NULL only *count is set. */
int pauli_jw_molecular_raw(int n_orb, const double *h, const double *g, double e_nn,
                           double eps_int, int64_t *count, uint64_t *x, uint64_t *z, double *c_re,
                           double *c_im);

/* Jordan-Wigner image of a sum of fermionic monomials
 *   sum_t c_t f_{t,0} f_{t,1} ... f_{t,nf_t - 1},  f = a_P (dagger 0) or a_P^dagger (1),
 * host arrays: n_factors[n_terms] (each 1..8), modes / daggers with all
 * factors back to back, c_re / c_im[n_terms].  Raw entries term by term in
 * expansion order, then canonical reduction.  Blocking. */
int pauli_jw_fermion(int n_qubits, int n_terms, const int *n_factors, const int *modes,
                     const int *daggers, const double *c_re, const double *c_im, double eps_drop,
                     pauli_sum **out);

/* Canonical form of the operator product A B (eq. pauli_operator_multiplication:
 * pairwise string products by eq. pauli_prod_x / pauli_prod_z /
 * pauli_prod_phase).  In XZ form the product of terms a_k and b_l is
 *   (Ca Cb (-1)^popcount(za & xb)) X^(xa ^ xb) Z^(za ^ zb);
 * the raw entries in the order k * M_B + l (complex products with separately
 * rounded parts, no fused multiply-add) are reduced as by pauli_sum_build.
 * PAULI_EUNSUPPORTED beyond 2^31 raw pairs.  Blocking. */
int pauli_sum_product(const pauli_sum *A, const pauli_sum *B, double eps_drop, pauli_sum **out);

/* Canonical form of A + beta B (A's terms, then B's scaled by beta, reduced
 * as by pauli_sum_build; e.g. beta = -1 for the commutator AB - BA of two
 * products).  Blocking. */
int pauli_sum_add(const pauli_sum *A, const pauli_sum *B, double beta_re, double beta_im, double eps_drop,
                  pauli_sum **out);

/* ------------------------------------------------------------------------- */
/* Pauli sums on more than 64 qubits (multi-word masks; operator algebra only) */
/* ------------------------------------------------------------------------- */

/* The same canonical form for up to 256 qubits, with masks of
 * W = ceil(n / 64) 64-bit words (word w holds qubits 64w .. 64w + 63; term t
 * has words x[t * W + w], z[t * W + w]) and (x, z) ordered as unsigned
 * multi-word integers, x first.  For the large Jordan-Wigner builds of
 * Sec. 3.1.1; state-vector calls take the 64-qubit pauli_sum. */
typedef struct pauli_wsum pauli_wsum;

/* pauli_jw_fermion for n_qubits <= 256 (same arguments, raw order and reduction). */
int pauli_wsum_jw_fermion(int n_qubits, int n_terms, const int *n_factors, const int *modes, const int *daggers,
                          const double *c_re, const double *c_im, double eps_drop, pauli_wsum **out);

/* pauli_jw_molecular for n_orb <= 128 (2 n_orb <= 256 qubits; same integral
 * layout, skipping rules, raw order and reduction). */
int pauli_wsum_jw_molecular(int n_orb, const double *h, const double *g, double e_nn, double eps_int,
                            double eps_drop, pauli_wsum **out);

/* pauli_sum_product for multi-word masks (PAULI_EUNSUPPORTED beyond 2^30 raw pairs). */
int pauli_wsum_product(const pauli_wsum *A, const pauli_wsum *B, double eps_drop, pauli_wsum **out);

int pauli_wsum_info(const pauli_wsum *h, int *n_qubits, int *words, int64_t *m, int64_t *n_groups);
/* host arrays x, z of M * W words, c_re, c_im of M */
int pauli_wsum_export(const pauli_wsum *h, uint64_t *x, uint64_t *z, double *c_re, double *c_im);
/* group_start[G + 1]: term offsets of the X-mask groups */
int pauli_wsum_groups(const pauli_wsum *h, int64_t *group_start);
int pauli_wsum_destroy(pauli_wsum *h);

/* Sizes: qubits, canonical terms M and X-mask groups G. */
int pauli_sum_info(const pauli_sum *h, int *n_qubits, int64_t *m, int64_t *n_groups);

/* Copy the canonical arrays (XZ-form coefficients) to host arrays of M entries. */
int pauli_sum_export(const pauli_sum *h, uint64_t *x, uint64_t *z, double *c_re, double *c_im);

/* Copy the X-mask group table to host arrays: group_x[G], group_start[G + 1]
 * (term offsets into the canonical arrays). */
int pauli_sum_groups(const pauli_sum *h, uint64_t *group_x, int64_t *group_start);

int pauli_sum_destroy(pauli_sum *h);

/* ------------------------------------------------------------------------- */
/* sectors (Sec. 2.4 spin-resolved product basis and symmetry blocks)        */
/* ------------------------------------------------------------------------- */

/* kind FULL: n_qubits <= 40, n_lo (1..min(n,24), 0 = default) only sets how
 * the kernels tile the index; k_lo / k_hi are ignored.  kind BLOCKS:
 * 1 <= n_lo < n_qubits, n_lo <= 24, n_qubits - n_lo <= 24, 1..33 blocks with
 * 0 <= k_lo <= n_lo, 0 <= k_hi <= n - n_lo and distinct k_hi.  Blocking. */
int pauli_sector_create(int n_qubits, int kind, int n_lo, int n_blocks, const int *k_lo,
                        const int *k_hi, pauli_sector **out);

/* A sector of abelian point-group blocks (Sec. 2.4: symmetry blocks r of
 * eq. sreverse_sum).  qubit_irrep[q] (0..7, n_qubits entries) labels every
 * qubit with an irrep of a group of order 8 whose product is XOR (e.g. D2h);
 * the irrep of a half string is the XOR of its occupied qubits' labels.  Block
 * r holds the configurations whose low n_lo qubits have k_lo[r] ones and
 * irrep irrep_lo[r] and whose high qubits have k_hi[r] ones and irrep
 * irrep_hi[r]; the (k_hi, irrep_hi) of the blocks must be distinct.  Inside a
 * block index = off_r + rank(b_hi) D_lo^r + rank(b_lo), rank = position in
 * ascending numeric order among the strings of the same (popcount, irrep).
 * Every apply / expect / rotate / pool / Krylov call takes these sectors;
 * pair-listed rotations and the rank-staged gathers of low halves wider than
 * 14 qubits fall back to the per-target kernels.  Blocking. */
int pauli_sector_create_irrep(int n_qubits, int n_lo, int n_blocks, const int *k_lo, const int *irrep_lo,
                              const int *k_hi, const int *irrep_hi, const int *qubit_irrep, pauli_sector **out);

int pauli_sector_dim(const pauli_sector *s, int64_t *dim);

/* Rank (configuration -> index, -1 if outside the sector) and unrank (index ->
 * configuration; out-of-range indices give all-ones) of n entries; device
 * arrays, enqueued on st.  Ranking uses the binomial table
 * rank(b) = sum_j C(p_j, j + 1) over the ascending set-bit positions p_j of
 * each half of b. */
int pauli_sector_rank(const pauli_sector *s, const uint64_t *configs, int64_t n, int64_t *idx,
                      pauli_stream_t st);
int pauli_sector_unrank(const pauli_sector *s, const int64_t *idx, int64_t n, uint64_t *configs,
                        pauli_stream_t st);

int pauli_sector_destroy(pauli_sector *s);

/* ------------------------------------------------------------------------- */
/* operator-state products (Sec. 2.4, eq. reverse_sum / sreverse_sum)        */
/* ------------------------------------------------------------------------- */

/* Build (and cache in H) the apply plan for this sector's split (allocates).
 * pauli_apply / pauli_expect build it on first use; call this first if the
 * later calls are to be captured in a CUDA graph.  Blocking. */
int pauli_prepare(pauli_sum *H, const pauli_sector *s);

/* psi_out = P_S H P_S psi_in (sources outside the sector count as zero):
 *   (H psi)_t = sum_g psi[t XOR x_g] * sum_{k in g} C_k (-1)^popcount(z_k & (t XOR x_g)),
 * gathered per target t without atomics.  psi_in and psi_out must not
 * overlap.  C64 accumulates group sums and amplitudes in FP32, C128 in FP64. */
int pauli_apply(pauli_sum *H, const pauli_sector *s, const void *psi_in, void *psi_out, int dtype,
                pauli_stream_t st);

/* result[0..3] (DEVICE, 4 doubles) = { Re <psi|H|psi>, Im <psi|H|psi>, ||H psi||^2, <psi|psi> }
 * (eq. vqe_energy), reduced in FP64 in a fixed order (deterministic).  If
 * hpsi_out is not NULL, H psi is also stored there (same dtype). */
int pauli_expect(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype, double *result,
                 void *hpsi_out, pauli_stream_t st);

/* pauli_expect without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot have device memory allocated on
 * their behalf -- programs whose GPU memory is entirely owned by another
 * allocator (a framework's caching pool that reserves the device), and
 * latency-critical loops where a cudaMalloc / cudaFree (which can synchronise
 * the whole device) is not acceptable.
 * Same arguments, results and precision as pauli_expect.  Its per-block
 * partial sums live in one static device array of 65,536 blocks x 4 doubles
 * (2 MiB, held on every GPU that loads the library until the process exits)
 * instead of memory the library allocates:
 *   - the plan for this sector's split must already exist: call
 *     pauli_prepare(H, s) (which allocates) once beforehand, otherwise
 *     PAULI_EINVAL;
 *   - a sector whose launch needs more than 65,536 blocks gets
 *     PAULI_EUNSUPPORTED (the 24-qubit (6a,6b) sector needs 924);
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process (a cudaDeviceReset in between is not supported);
 *     make that first call before any stream capture;
 *   - a full-space sector of a lattice operator that is applied in passes over
 *     local bit sets (pauli_set_launch_config direct = 2, the default from 21
 *     qubits) accumulates H psi in a vector: there hpsi_out must be given,
 *     unless an earlier pauli_expect without it has already made the
 *     operator's own scratch vector; otherwise PAULI_EUNSUPPORTED;
 *   - every call uses the same array, and each block overwrites its own
 *     partials before they are read, so no state from an earlier call
 *     matters; calls that overlap on the GPU (different streams, no ordering
 *     between them) race on the array and must not be issued.
 * It calls no cudaMalloc, cudaFree or other allocating routine. */
int pauli_expect_noalloc(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype,
                         double *result, void *hpsi_out, pauli_stream_t st);

/* Selected rows of H psi: the target-driven gather of eq. reverse_sum
 * evaluated only at the n_rows target indices rows[0..n_rows) (DEVICE int64,
 * sector indices in [0, dim), distinct), one CTA per target, every group of H
 * in a fixed order.
 *   hpsi_out (DEVICE state vector of dim entries, or NULL): entry rows[i]
 *     <- (H psi)[rows[i]]; every other entry is left as it is.
 *   result (DEVICE, 4 doubles, or NULL): { Re, Im of sum_i conj(psi[r_i])
 *     (H psi)[r_i], sum_i |(H psi)[r_i]|^2, sum_i |psi[r_i]|^2 }, FP64 in a
 *     fixed order.  When psi vanishes outside the listed rows (a state that
 *     lives on a known set of configurations, e.g. the seniority-zero strings
 *     a pair-double ansatz reaches from a closed-shell reference), result[0]
 *     and result[1] are <psi|H|psi> exactly as pauli_expect gives them, and
 *     hpsi_out holds the part of H psi on those rows (all that the adjoint
 *     gradient of such a state needs).
 * At least one of hpsi_out and result must be given.  Precision as
 * pauli_apply (C64: FP32 group sums, C128: FP64).  An index outside [0, dim)
 * is skipped (nothing read or written for it, zero partials) and sets H's
 * device status word to PAULI_EINVAL (pauli_status).  The first call with
 * result, and any call with more rows than before, allocates the operator's
 * partial-sum buffer (n_rows x 4 doubles; synchronises st). */
int pauli_expect_rows(pauli_sum *H, const pauli_sector *s, const void *psi, int dtype, const int64_t *rows,
                      int64_t n_rows, void *hpsi_out, double *result, pauli_stream_t st);

/* psi <- exp(-i theta G) psi in place, for a Hermitian G with ONE X mask x
 * (a single group; Sec. 2.5 and the Trotter factors exp(theta tau) of
 * Sec. 3.2 with G = i tau).  G maps each pair {t, t XOR x} onto itself with
 * (G psi)_t = f_t psi_{t XOR x}, f_{t XOR x} = conj(f_t), so
 *   psi'_t = cos(theta |f_t|) psi_t - i sin(theta |f_t|) f_t / |f_t| psi_{t XOR x}
 * (x = 0: psi'_t = exp(-i theta f_t) psi_t).  PAULI_EINVAL if G has more than
 * one X mask, PAULI_ENOTHERMITIAN if a letter-form coefficient has an
 * imaginary part above 1e-12 max|C|.  If some t in the sector has
 * t XOR x outside it with f_t != 0, the device status word of G gets
 * PAULI_ESECTOR (see pauli_status) and those amplitudes are left unchanged.
 * On a single-product-block sector the first rotation by G checks that once
 * (synchronising st; make that first call outside stream capture) and, if G
 * keeps the sector, builds a list of the pairs {t, t XOR x} inside it; later
 * rotations visit only those pairs.  pauli_rotate_adjoint shares the list. */
int pauli_rotate(pauli_sum *G, const pauli_sector *s, double theta, void *psi, int dtype,
                 pauli_stream_t st);

/* One step of the adjoint (reverse-mode) gradient of a product ansatz
 * psi(theta) = U_K ... U_1 psi_0, U_k = exp(-i theta_k G_k) (Sec. 3.2):
 * result[0] + i result[1] = <lam|G|phi> from the input vectors (FP64,
 * fixed reduction order; result is a DEVICE array of 2 doubles), then
 * phi <- exp(-i theta G) phi and lam <- exp(-i theta G) lam in place, in one
 * pass over both vectors.  With phi = psi(theta), lam = H psi(theta) and
 * k = K..1 called with theta = -theta_k, dE/dtheta_k = 2 Im result_k.
 * Same generator rules and sector-leak status as pauli_rotate; phi != lam.
 * Uses the per-device scratch of pauli_vdot (see there). */
int pauli_rotate_adjoint(pauli_sum *G, const pauli_sector *s, double theta, void *phi, void *lam, int dtype,
                         double *result, pauli_stream_t st);

/* psi <- exp(-i theta_{k-1} G_{k-1}) ... exp(-i theta_0 G_0) psi: k calls of
 * pauli_rotate in order (a product-form ansatz, Sec. 3.2); stops at the first
 * error and returns it.  Gs: host array of k handles, thetas: host array. */
int pauli_rotate_seq(pauli_sum *const *Gs, const double *thetas, int k, const pauli_sector *s, void *psi,
                     int dtype, pauli_stream_t st);

/* A fixed product of single-group rotations (a Trotterised UCCSD / UCCGSD
 * step or any product ansatz, Sec. 3.2), applied tile by tile:
 *   psi <- exp(-i theta_{K-1} G_{K-1}) ... exp(-i theta_0 G_0) psi,
 * every G_k with pauli_rotate's generator rules (results equal K pauli_rotate
 * calls up to rounding; a generator that leaks out of the sector sets its
 * status word as there).  On a single product block, consecutive generators
 * are grouped into runs that share a tile -- generators with x_hi = 0 (and
 * diagonal ones) into tiles of one row, generators with x_lo = 0 into tiles of
 * all rows of a few adjacent columns, generators with one common nonzero x_hi
 * (with row-local and diagonal ones) into tiles of the two rows r and
 * r ^ x_hi -- and one launch per run reads and writes each tile once,
 * applying the run's rotations in order in shared memory.  Runs whose tile
 * exceeds shared memory, and sectors that are not one block, use one
 * pauli_rotate launch per generator.  The generators and the sector must
 * outlive the handle.  pauli_rotseq_create is blocking. */
typedef struct pauli_rotseq pauli_rotseq;
int pauli_rotseq_create(pauli_sum *const *Gs, int K, const pauli_sector *s, pauli_rotseq **out);

/* thetas: HOST array of K angles, copied into the handle on st (calls with one
 * handle must be ordered on one stream).  psi: device vector of the sector. */
int pauli_rotseq_apply(pauli_rotseq *q, const double *thetas, void *psi, int dtype, pauli_stream_t st);

/* Launches one apply makes in dtype, and how many generators run fused. */
int pauli_rotseq_info(const pauli_rotseq *q, int dtype, int *launches, int *fused);
int pauli_rotseq_destroy(pauli_rotseq *q);

/* result[0] + i result[1] = <x|y> = sum_i conj(x_i) y_i over n amplitudes of
 * type dtype, accumulated in FP64 in a fixed order (the same inputs give the
 * same bits); result is a DEVICE array of 2 doubles written on st.  x, y
 * 16-byte aligned device vectors (may be NULL if n == 0).  The per-block partial sums go to one
 * scratch array per device (8 x 4 doubles per SM), allocated on the first
 * call and kept until exit and shared with pauli_rotate_adjoint: calls of the
 * two issued on different streams must be ordered with events. */
int pauli_vdot(const void *x, const void *y, int64_t n, int dtype, double *result, pauli_stream_t st);

/* ------------------------------------------------------------------------- */
/* operator-pool gradients (operator selection of ADAPT-VQE, Sec. 3.3)        */
/* ------------------------------------------------------------------------- */

/* A pool of K Hermitian single-X-group generators G_k (pauli_rotate's
 * generator rules; the paper's anti-Hermitian pool operators are A_k = -i G_k)
 * on one sector.  pauli_pool_create checks every generator (PAULI_EINVAL: more
 * than one X mask; PAULI_ENOTHERMITIAN), builds or reuses each generator's
 * pair list on a single-block sector (a one-time leak check per generator, as
 * for pauli_rotate) and copies the tables, masks and coefficients into the
 * pool, so the generators may be destroyed afterwards; the sector must outlive
 * the pool.  Blocking. */
typedef struct pauli_pool pauli_pool;
int pauli_pool_create(pauli_sum *const *Gs, int K, const pauli_sector *s, pauli_pool **out);
int pauli_pool_size(const pauli_pool *p, int *K);

/* grads[k] = d/dtheta <psi| exp(i theta G_k) H exp(-i theta G_k) |psi> at 0
 *          = i <psi|[G_k, H]|psi> = 2 Im <hpsi|G_k psi> = <psi|[H, A_k]|psi>,
 * for every generator, given hpsi = H psi (the vector pauli_expect stores) on
 * the pool's sector: G_k acts as P_S G_k P_S (a generator that moves amplitude
 * out of the sector has its status word set to PAULI_ESECTOR, as in
 * pauli_rotate).  grads is a DEVICE array of K doubles; psi, hpsi are device
 * vectors of the sector's dimension in dtype, 16-byte aligned.  One launch
 * contracts every pair-listed generator; each gradient is an FP64 sum in a
 * fixed order (the same inputs give the same bits). */
int pauli_pool_gradients(pauli_pool *p, const void *psi, const void *hpsi, int dtype, double *grads,
                         pauli_stream_t st);
int pauli_pool_destroy(pauli_pool *p);

/* ------------------------------------------------------------------------- */
/* learned warm start: a small multilayer perceptron on the tensor cores      */
/* ------------------------------------------------------------------------- */

/* y = W3^T tanh(W2^T tanh(W1^T x + b1) + b2) + b3 mapping a geometry
 * descriptor (in_dim values, e.g. a bond length) to the out_dim ansatz
 * amplitudes that start the variational optimisation at that geometry
 * (the learned warm start of Sec. 4).  The two hidden-width products run in
 * BF16 on the tensor cores with FP32 accumulation; master weights, biases,
 * the first layer and Adam are FP32.  Parameter vector layout (FP32):
 * W1[in][hid], b1[hid], W2[hid][hid], b2[hid], W3[hid][out], b3[out],
 * row-major, W[k][j] multiplying input k into output j.  A new network has
 * all parameters zero; set them with pauli_mlp_set_params. */
typedef struct pauli_mlp pauli_mlp;
int pauli_mlp_create(int in_dim, int hidden, int out_dim, int max_batch, pauli_mlp **out);
int pauli_mlp_num_params(const pauli_mlp *m, int64_t *n);
/* host <-> device copies of the parameter vector (set also zeroes Adam's moments); blocking */
int pauli_mlp_set_params(pauli_mlp *m, const float *params);
int pauli_mlp_get_params(const pauli_mlp *m, float *params);

/* y[batch][out] = net(x[batch][in]); x, y DEVICE FP32 arrays; 1 <= batch <= max_batch */
int pauli_mlp_forward(pauli_mlp *m, int batch, const float *x, float *y, pauli_stream_t st);

/* Forward pass, loss = 1/(2 batch) sum (y - target)^2 (device double, if loss
 * is not NULL) and its gradient with respect to every parameter, kept in the
 * handle for pauli_mlp_adam_step and copied to the DEVICE array grads (same
 * layout as the parameters) if grads is not NULL. */
int pauli_mlp_backward(pauli_mlp *m, int batch, const float *x, const float *target, float *grads,
                       double *loss, pauli_stream_t st);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for step
 * t >= 1) with the gradient of the last pauli_mlp_backward. */
int pauli_mlp_adam_step(pauli_mlp *m, float lr, int t, pauli_stream_t st);

/* steps x (pauli_mlp_backward + pauli_mlp_adam_step with t = t0+1 .. t0+steps)
 * in one call, enqueued on st; loss (device double, may be NULL) is that of
 * the last step's forward pass.  The first steps - 1 steps replay a CUDA graph
 * of one step (captured on the handle's own stream on the first call and again
 * whenever batch, x, target or lr change; ordered after and before st with
 * events), the last one runs directly on st; the arithmetic is that of the
 * eager steps.  Calls with one handle must be ordered; st must not itself be
 * under stream capture. */
int pauli_mlp_train(pauli_mlp *m, int batch, const float *x, const float *target, int steps, float lr, int t0,
                    double *loss, pauli_stream_t st);

int pauli_mlp_destroy(pauli_mlp *m);

/* ------------------------------------------------------------------------- */
/* launch-shape autotuning                                                    */
/* ------------------------------------------------------------------------- */

/* Launch shape of pauli_apply / pauli_expect for one (operator, sector, dtype):
 * columns (targets) per thread, staged source rows in flight, piece ranges a
 * row is split into (their partial vectors are added in a fixed order),
 * direct gather (operators small enough to keep whole in shared memory) vs
 * staged source rows vs, in the full space, passes over local bit sets (each
 * pass stages 2^13-amplitude chunks that contain every X mask of its groups),
 * vs, in a single-block sector with a low half of at most 12 qubits, a gather
 * over per-item lists of the (target, source) pairs that stay in the block
 * (one thread block per row, warp-private accumulator rows in shared memory),
 * and (single-block sectors) rows staged densely by rank with a rank table vs
 * by bit pattern.  ms: measured time of one apply (0 if
 * not measured). */
typedef struct {
    int cols_per_thread;  /* 1, 2 or 4; 8 with rank-staged rows (else used as 4) */
    int staged_rows;      /* 1 or 2 */
    int row_split;        /* 1..16 */
    int direct;           /* 0 staged rows, 1 direct gather (small operators),
                             2 full space in passes over local bit sets (lattice operators),
                             3 lists of valid pairs (single block, low half <= 12 qubits),
                             4 SVD-factorised phases (real operator, single block; see
                               pauli_svd_ranks) */
    int ranked;           /* 0 or 1 */
    double ms;
} pauli_launch_config;

/* Times every realisable shape (reps launches each, CUDA events on st, after
 * one warm-up launch, on scratch vectors the call allocates) and keeps the
 * fastest in H for this sector and dtype; later applies use it.  Blocking. */
int pauli_tune(pauli_sum *H, const pauli_sector *s, int dtype, int reps, pauli_launch_config *best,
               pauli_stream_t st);

/* Installs a shape (e.g. read back from a cache of earlier pauli_tune results). */
int pauli_set_launch_config(pauli_sum *H, const pauli_sector *s, int dtype, const pauli_launch_config *cfg);

/* The shape pauli_apply currently uses for this sector and dtype (needs a plan). */
int pauli_get_launch_config(pauli_sum *H, const pauli_sector *s, int dtype, pauli_launch_config *cfg);

/* The gather of eq. svd_sreverse_sum (Sec. 2.4, Algorithm 2), installed with
 * direct = 4 (cols_per_thread 1, 2 or 4) or chosen by pauli_tune: for every
 * X-mask group the matrix M_{mu nu} of its coefficients over its distinct
 * (low, high) Z-mask pairs is factorised by SVD (one-sided Jacobi, FP64,
 * singular values above 1e-12 kept), M = sum_k Wa_k Wb_k^T, so that its phase
 * sum at a target is sum_k Fa(t_lo, k) Fb(t_hi, k).  Fb is evaluated once per
 * (row, group) and Fa is tabulated for the low half in on-the-fly batches of
 * groups (at most 256 MB of table at a time); a batch after the first adds to
 * the output, so an expectation without hpsi_out on an operator that needs
 * several batches returns PAULI_EUNSUPPORTED.  Needs a real operator on a
 * single product block with a low half of at most 16 qubits
 * (PAULI_EUNSUPPORTED otherwise).  pauli_svd_ranks builds the factorisation
 * if needed (blocking) and reports hist[R] = number of groups of rank R
 * (R < len; groups whose coefficients all cancel have rank 0) and the number
 * of on-the-fly batches. */
int pauli_svd_ranks(pauli_sum *H, const pauli_sector *s, int *hist, int len, int *batches);

/* Cache of tuned shapes in a text file (one line per (operator, sector,
 * dtype): a tag, a key, the dtype and the five fields and ms of
 * pauli_launch_config).  The key is the device name, the sector's shape
 * (qubits, split, kind, blocks, dimension), the operator's term and group
 * counts and a 64-bit FNV-1a hash of its canonical arrays, so an entry is only
 * installed on the operator and sector it was measured for.
 * pauli_tune_save writes the shapes tuned or installed for (H, s) -- both
 * dtypes, where present -- replacing earlier lines with the same key and
 * dtype (the file is rewritten through a temporary file and a rename; writers
 * of one file must not run concurrently).  pauli_tune_load installs every
 * matching entry with pauli_set_launch_config and sets *found to their
 * number (0 if the file does not exist).  Both need a plan (pauli_prepare)
 * and are blocking.  Errors: PAULI_EINVAL for bad handles, a NULL path or an
 * unwritable file. */
int pauli_tune_save(pauli_sum *H, const pauli_sector *s, const char *path);
int pauli_tune_load(pauli_sum *H, const pauli_sector *s, const char *path, int *found);

/* ------------------------------------------------------------------------- */
/* many independent states in one persistent launch                           */
/* ------------------------------------------------------------------------- */

/* A batch of n (operator, sector) pairs -- e.g. the points of a scan or the
 * parameter-shifted states of a gradient -- applied together in persistent
 * launches: a grid of resident CTAs pulls (state, row, column tile) work
 * units from an atomic queue, largest states first.  By default every state
 * keeps the staged-gather shape a launch of its own would take, and the
 * states of one shape share one persistent launch (one launch per distinct
 * shape); a uniform shape can be installed or tuned instead.  Every sector
 * must be a single product block; the handles must outlive the batch;
 * pauli_batch_create calls pauli_prepare on each pair. */
typedef struct pauli_batch pauli_batch;
int pauli_batch_create(int n, pauli_sum *const *H, const pauli_sector *const *S, int dtype,
                       pauli_batch **out);

/* For every state b: psi_out[b] = H_b psi_in[b] (skipped if psi_out is NULL
 * or psi_out[b] is NULL) and, if results is not NULL, results[4b..4b+3] =
 * { Re <psi|H|psi>, Im <psi|H|psi>, ||H psi||^2, <psi|psi> } (DEVICE array,
 * FP64, fixed reduction order).  psi_in / psi_out are HOST arrays of n device
 * pointers.  The only atomic is the work-queue counter. */
int pauli_batch_apply(pauli_batch *b, const void *const *psi_in, void *const *psi_out, double *results,
                      pauli_stream_t st);

/* Times the per-state shapes and every uniform columns-per-thread /
 * staged-rows / staging layout on the given vectors and keeps the fastest
 * (best->cols_per_thread = 0 for the per-state shapes).  Blocking. */
int pauli_batch_tune(pauli_batch *b, const void *const *psi_in, void *const *psi_out, int reps,
                     pauli_launch_config *best, pauli_stream_t st);

/* Installs a uniform launch shape for the batch (cols_per_thread 1, 2 or 4,
 * staged_rows 1 or 2, ranked 0 or 1; row_split must be 1 and direct 0), or,
 * with cols_per_thread = 0, goes back to the per-state shapes:
 * PAULI_EUNSUPPORTED if the staging layout does not fit in shared memory for
 * the widest state.  pauli_batch_get_launch_config reads the shape in use
 * (cols_per_thread = 0 for per-state shapes; ms = launches per apply). */
int pauli_batch_set_launch_config(pauli_batch *b, const pauli_launch_config *cfg);
int pauli_batch_get_launch_config(const pauli_batch *b, pauli_launch_config *cfg);

int pauli_batch_destroy(pauli_batch *b);

/* ------------------------------------------------------------------------- */
/* real-time propagation by Krylov (Lanczos) projection                       */
/* ------------------------------------------------------------------------- */

/* psi <- exp(-i dt H) psi on the sector for a Hermitian H, by an m-vector
 * Lanczos projection (the paper names Krylov solvers as users of the same
 * operator engine, Sec. 4): v_0 = psi/||psi||, w_j = H v_j, alpha_j = <v_j|w_j>,
 * w_j -= alpha_j v_j + beta_j v_{j-1}, beta_{j+1} = ||w_j||, v_{j+1} = w_j/beta_{j+1},
 * psi = ||psi|| V_m exp(-i dt T_m) e_0.  Vectors are stored in dtype; alpha,
 * beta and the m x m exponential (cyclic Jacobi eigen-decomposition of T_m)
 * are FP64 and stay on the device.  2 <= m <= 32.  The handle owns
 * (m+1) x dim vectors of scratch (pauli_krylov_create allocates them and
 * calls pauli_prepare).  A zero w_j (invariant subspace) gives zero later
 * vectors and an exact result. */
typedef struct pauli_krylov pauli_krylov;
int pauli_krylov_create(pauli_sum *H, const pauli_sector *s, int m, int dtype, pauli_krylov **out);

/* nsteps propagation steps of length dt on st.  use_graph != 0: the step is
 * captured once as a CUDA graph (after one eager step, re-captured when psi,
 * dt or st change) and replayed, so a step makes no host round trip. */
int pauli_krylov_step(pauli_krylov *k, void *psi, double dt, int nsteps, int use_graph,
                      pauli_stream_t st);

/* Copies the last step's alpha[m] and beta[m+1] (beta[0] = ||psi||) to host
 * arrays; synchronizes st. */
int pauli_krylov_scalars(const pauli_krylov *k, double *alpha, double *beta, pauli_stream_t st);

int pauli_krylov_destroy(pauli_krylov *k);

/* Reads and clears H's device status word; synchronizes st.  *code is
 * PAULI_OK or the first device-side error recorded since the last read. */
int pauli_status(pauli_sum *H, pauli_stream_t st, int *code);

#ifdef __cplusplus
}
#endif
#endif /* PAULISIM_H */
