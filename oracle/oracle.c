/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the Pauli-algebra operator-state path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline / reference legs may load this library.  It shares no
 * code, header, table or constant with the CUDA library; the two meet only in
 * the seeded input arrays of workloads/.
 *
 * Every routine writes out the plain definition of what it computes, in the
 * paper's notation, with no blocking, fusion or reordering:
 *
 *   letters and products  Sec. 2.2 (eq. single_pauli_mapping, eq. pauli_group):
 *                         per-qubit textbook table XY = iZ, YZ = iX, ZX = iY,
 *                         reversed order gives -i; the string phase is an
 *                         integer mod 4.  (The bitwise rule of
 *                         eq. pauli_prod_phase is NOT used here.)
 *   symplectic form       Sec. 2.2.2 / 2.3: C = c * i^(gamma + #Y), #Y = popcnt(X & Z),
 *                         so a letter string equals i^#Y X^x Z^z.
 *   Jordan-Wigner         Sec. 2.3, eq. for a_p^dagger / a_p and Algorithm 1: each
 *                         ladder operator is a sum of two letter strings; a
 *                         one-/two-body term is the product of 2 / 4 of them
 *                         (4 / 16 raw entries), in a fixed raw order.
 *   canonical reduction   Sec. 2.3: unique strings sorted by (X, Z) as unsigned
 *                         integers, coefficients accumulated in raw order,
 *                         terms with |C|^2 <= eps^2 dropped.
 *   sector                Sec. 2.4 (spin-resolved product basis, symmetry
 *                         blocks) and eq. fcidim: explicit enumeration; the
 *                         index of a configuration is its position in that list.
 *   apply                 eq. grouped_contraction in SOURCE form, term by term
 *                         (no grouping): out[t] += C_k (-1)^popc(Z_k & s) psi[s]
 *                         for t = s XOR X_k.  A per-target form
 *                         <t|H|psi> = sum_k C_k <t|P_k|psi> serves sampled rows.
 *   expectation           eq. vqe_energy: E = sum_t conj(psi_t) (H psi)_t.
 *   rotation              exp(-i theta G) psi by its Taylor series, applied with
 *                         the source-form apply above (Sec. 2.5 / Sec. 3.2's
 *                         Trotter factors exp(theta tau), G = i tau).
 *   Hartree-Fock energy   Slater-Condon closed form for the determinant with
 *                         the lowest N_alpha / N_beta orbitals occupied.
 *
 * Compile with -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------- */
/* complex helpers (explicit, no fused multiply-add)                          */
/* ------------------------------------------------------------------------- */
typedef struct { double re, im; } cplx;

static cplx c_make(double re, double im) { cplx r; r.re = re; r.im = im; return r; }
static cplx c_add(cplx a, cplx b) { return c_make(a.re + b.re, a.im + b.im); }
static cplx c_mul(cplx a, cplx b)
{
    double rr = a.re * b.re;
    double ii = a.im * b.im;
    double ri = a.re * b.im;
    double ir = a.im * b.re;
    return c_make(rr - ii, ri + ir);
}
static cplx c_scale(cplx a, double s) { return c_make(a.re * s, a.im * s); }
/* multiply by i^k exactly (a rotation by a quarter turn is a swap and a sign) */
static cplx c_ipow(cplx a, int k)
{
    k &= 3;
    if (k == 0) return a;
    if (k == 1) return c_make(-a.im, a.re);
    if (k == 2) return c_make(-a.re, -a.im);
    return c_make(a.im, -a.re);
}

static int popc64(uint64_t v)
{
    int c = 0;
    while (v) { c += (int)(v & 1u); v >>= 1; }
    return c;
}

/* ------------------------------------------------------------------------- */
/* single-qubit letters, eq. single_pauli_mapping                             */
/* ------------------------------------------------------------------------- */
enum { L_I = 0, L_X = 1, L_Y = 2, L_Z = 3 };

/* Letter from the bit pair (a, b) via the type-recovery relations
 * T_y = a AND b, T_x = a XOR T_y, T_z = b XOR T_y. */
static int letter_of(int a, int b)
{
    int ty = a & b;
    int tx = a ^ ty;
    int tz = b ^ ty;
    if (ty) return L_Y;
    if (tx) return L_X;
    if (tz) return L_Z;
    return L_I;
}

static void bits_of(int letter, int *a, int *b)
{
    *a = (letter == L_X || letter == L_Y);
    *b = (letter == L_Y || letter == L_Z);
}

/* Textbook products sigma_u sigma_v = i^k sigma_w, written out in full. */
static const int MUL_W[4][4] = {
    /*        I    X    Y    Z  */
    /* I */ {L_I, L_X, L_Y, L_Z},
    /* X */ {L_X, L_I, L_Z, L_Y},
    /* Y */ {L_Y, L_Z, L_I, L_X},
    /* Z */ {L_Z, L_Y, L_X, L_I},
};
static const int MUL_K[4][4] = {
    /*       I  X  Y  Z        XY = iZ, XZ = -iY, YX = -iZ, YZ = iX, ZX = iY, ZY = -iX */
    /* I */ {0, 0, 0, 0},
    /* X */ {0, 0, 1, 3},
    /* Y */ {0, 3, 0, 1},
    /* Z */ {0, 1, 3, 0},
};

int orc_letter_mul(int u, int v, int *k)
{
    *k = MUL_K[u][v];
    return MUL_W[u][v];
}

/* Product of two LETTER strings (x, z masks in the letter sense), qubit by
 * qubit.  Returns the letter string of the product in (x, z) and the phase
 * i^k, k mod 4. */
void orc_string_mul(int n, uint64_t xa, uint64_t za, uint64_t xb, uint64_t zb,
                    uint64_t *x, uint64_t *z, int *k)
{
    uint64_t ox = 0, oz = 0;
    int ph = 0;
    for (int q = 0; q < n; ++q) {
        int u = letter_of((int)((xa >> q) & 1u), (int)((za >> q) & 1u));
        int v = letter_of((int)((xb >> q) & 1u), (int)((zb >> q) & 1u));
        int kk;
        int w = orc_letter_mul(u, v, &kk);
        int a, b;
        bits_of(w, &a, &b);
        ox |= (uint64_t)a << q;
        oz |= (uint64_t)b << q;
        ph += kk;
    }
    *x = ox;
    *z = oz;
    *k = ph & 3;
}

/* Number of Y letters of a letter string: qubits with both bits set. */
static int count_y(int n, uint64_t x, uint64_t z)
{
    int c = 0;
    for (int q = 0; q < n; ++q)
        if (letter_of((int)((x >> q) & 1u), (int)((z >> q) & 1u)) == L_Y) ++c;
    return c;
}

/* Convert m terms to symplectic (XZ) form: C = i^gamma * c * (letter ? i^#Y : 1). */
void orc_to_xz(int n, int64_t m, const uint64_t *x, const uint64_t *z, const uint8_t *gamma,
               const double *cre, const double *cim, int letter_form, double *ore, double *oim)
{
    for (int64_t j = 0; j < m; ++j) {
        cplx c = c_make(cre[j], cim[j]);
        int k = gamma ? (int)gamma[j] : 0;
        if (letter_form) k += count_y(n, x[j], z[j]);
        c = c_ipow(c, k);
        ore[j] = c.re;
        oim[j] = c.im;
    }
}

/* ------------------------------------------------------------------------- */
/* Jordan-Wigner raw entries (Sec. 2.3, Algorithm 1)                          */
/* ------------------------------------------------------------------------- */
/* A ladder operator on spin orbital P is the two-term letter sum
 *   a_P^dagger = 1/2 X_P Z_{<P} - i/2 Y_P Z_{<P},
 *   a_P        = 1/2 X_P Z_{<P} + i/2 Y_P Z_{<P}.
 * Term 0 is the X version, term 1 the Y version. */
typedef struct { uint64_t x, z; cplx c; } lterm;

static void ladder(int P, int dagger, lterm out[2])
{
    uint64_t below = (P == 0) ? 0 : ((((uint64_t)1) << P) - 1);
    uint64_t bit = ((uint64_t)1) << P;
    out[0].x = bit; out[0].z = below;       out[0].c = c_make(0.5, 0.0);
    out[1].x = bit; out[1].z = below | bit; out[1].c = c_make(0.0, dagger ? -0.5 : 0.5);
}

/* Expand the product of nf ladder operators (left to right) into 2^nf letter
 * strings, entry order = expansion index with the LEFT factor most significant,
 * multiply by `scale`, convert to XZ form and append to the output arrays. */
static int64_t expand_product(int n, const lterm *f[], int nf, cplx scale, int64_t pos,
                              uint64_t *ox, uint64_t *oz, double *ore, double *oim)
{
    int ne = 1 << nf;
    for (int e = 0; e < ne; ++e) {
        uint64_t x = 0, z = 0;
        cplx c = c_make(1.0, 0.0);
        int ph = 0;
        for (int j = 0; j < nf; ++j) {
            int sel = (e >> (nf - 1 - j)) & 1;
            const lterm *t = &f[j][sel];
            uint64_t nx, nz;
            int k;
            orc_string_mul(n, x, z, t->x, t->z, &nx, &nz, &k);
            x = nx; z = nz; ph += k;
            c = c_mul(c, t->c);
        }
        c = c_ipow(c, ph);
        c = c_mul(c, scale);
        /* letter form -> XZ form */
        c = c_ipow(c, count_y(n, x, z));
        if (ox) {
            ox[pos] = x; oz[pos] = z; ore[pos] = c.re; oim[pos] = c.im;
        }
        ++pos;
    }
    return pos;
}

/* H = sum_{sigma,pq} h_pq a+_{p sigma} a_{q sigma}
 *   + 1/2 sum_{sigma tau, pqrs} (pq|rs) a+_{p sigma} a+_{r tau} a_{s tau} a_{q sigma}
 * with spin orbital P = p (alpha) or norb + p (beta).  An integral is used when
 * |value| > eps (strict).  Two-body terms with P == R or Q == S vanish
 * identically and are skipped.
 * Raw order: one-body (sigma, p, q ascending, 4 entries each), then two-body
 * (sigma, tau, p, q, r, s ascending, 16 entries each).
 * Returns the number of raw entries; arrays may be NULL to count only. */
int64_t orc_jw_raw(int norb, const double *h, const double *g, double eps,
                   uint64_t *ox, uint64_t *oz, double *ore, double *oim)
{
    int n = 2 * norb;
    int64_t pos = 0;
    lterm A[2], B[2], Cq[2], Dq[2];
    for (int sg = 0; sg < 2; ++sg)
        for (int p = 0; p < norb; ++p)
            for (int q = 0; q < norb; ++q) {
                double v = h[p * norb + q];
                if (!(fabs(v) > eps)) continue;
                ladder(sg * norb + p, 1, A);
                ladder(sg * norb + q, 0, B);
                const lterm *f[2] = {A, B};
                pos = expand_product(n, f, 2, c_make(v, 0.0), pos, ox, oz, ore, oim);
            }
    for (int sg = 0; sg < 2; ++sg)
        for (int tu = 0; tu < 2; ++tu)
            for (int p = 0; p < norb; ++p)
                for (int q = 0; q < norb; ++q)
                    for (int r = 0; r < norb; ++r)
                        for (int s = 0; s < norb; ++s) {
                            int P = sg * norb + p, Q = sg * norb + q;
                            int R = tu * norb + r, S = tu * norb + s;
                            if (P == R || Q == S) continue;
                            double v = g[((p * norb + q) * norb + r) * norb + s];
                            if (!(fabs(v) > eps)) continue;
                            ladder(P, 1, A);
                            ladder(R, 1, B);
                            ladder(S, 0, Cq);
                            ladder(Q, 0, Dq);
                            const lterm *f[4] = {A, B, Cq, Dq};
                            pos = expand_product(n, f, 4, c_make(0.5 * v, 0.0), pos, ox, oz, ore, oim);
                        }
    return pos;
}

/* Raw entries of a sum of fermionic monomials sum_t c_t f_{t,0} f_{t,1} ...
 * (each factor a_P or a_P^dagger, left to right), term by term in input
 * order, 2^nf entries per term in expansion order.  modes / dag hold the
 * factors of all terms back to back; nf[t] is the factor count of term t
 * (at most 8).  Returns the entry count; arrays may be NULL to count only. */
int64_t orc_fermion_raw(int n, int nterms, const int *nf, const int *modes, const int *dag,
                        const double *cre, const double *cim, uint64_t *ox, uint64_t *oz,
                        double *ore, double *oim)
{
    int64_t pos = 0;
    int at = 0;
    lterm fac[8][2];
    for (int t = 0; t < nterms; ++t) {
        const lterm *f[8];
        for (int j = 0; j < nf[t]; ++j) {
            ladder(modes[at + j], dag[at + j], fac[j]);
            f[j] = fac[j];
        }
        pos = expand_product(n, f, nf[t], c_make(cre[t], cim[t]), pos, ox, oz, ore, oim);
        at += nf[t];
    }
    return pos;
}

/* The two letter strings of a ladder operator in XZ form (x, z, C). */
void orc_jw_ladder(int P, int dagger, uint64_t *ox, uint64_t *oz, double *ore, double *oim)
{
    lterm t[2];
    ladder(P, dagger, t);
    for (int j = 0; j < 2; ++j) {
        cplx c = c_ipow(t[j].c, count_y(64, t[j].x, t[j].z));
        ox[j] = t[j].x; oz[j] = t[j].z; ore[j] = c.re; oim[j] = c.im;
    }
}

/* Raw product of two Pauli sums in XZ form (eq. pauli_operator_multiplication
 * as a definition): every pair (k, l), k outer, becomes one entry.  Each XZ
 * string is turned back into its letter string (divide by i^#Y), the letter
 * strings are multiplied qubit by qubit, and the result is put in XZ form
 * again.  Output arrays hold ma * mb entries. */
void orc_sum_product(int n, int64_t ma, const uint64_t *xa, const uint64_t *za, const double *ra,
                     const double *ia, int64_t mb, const uint64_t *xb, const uint64_t *zb,
                     const double *rb, const double *ib, uint64_t *ox, uint64_t *oz, double *ore,
                     double *oim)
{
    int64_t pos = 0;
    for (int64_t k = 0; k < ma; ++k)
        for (int64_t l = 0; l < mb; ++l) {
            cplx ca = c_ipow(c_make(ra[k], ia[k]), 4 - (count_y(n, xa[k], za[k]) & 3));
            cplx cb = c_ipow(c_make(rb[l], ib[l]), 4 - (count_y(n, xb[l], zb[l]) & 3));
            uint64_t x, z;
            int ph;
            orc_string_mul(n, xa[k], za[k], xb[l], zb[l], &x, &z, &ph);
            cplx c = c_ipow(c_mul(ca, cb), ph + count_y(n, x, z));
            ox[pos] = x; oz[pos] = z; ore[pos] = c.re; oim[pos] = c.im;
            ++pos;
        }
}

/* ------------------------------------------------------------------------- */
/* canonical reduction (Sec. 2.3)                                             */
/* ------------------------------------------------------------------------- */
/* (x, z) key order of entries a and b (keys passed in: the sort holds no
 * global state, so calls from several threads do not interfere) */
static int key_less(const uint64_t *kx, const uint64_t *kz, int64_t a, int64_t b)
{
    if (kx[a] != kx[b]) return kx[a] < kx[b];
    return kz[a] < kz[b];
}

/* plain top-down stable merge sort of an index array by the (x, z) key */
static void msort(const uint64_t *kx, const uint64_t *kz, int64_t *idx, int64_t *tmp, int64_t n)
{
    if (n < 2) return;
    int64_t h = n / 2;
    msort(kx, kz, idx, tmp, h);
    msort(kx, kz, idx + h, tmp, n - h);
    int64_t i = 0, j = h, k = 0;
    while (i < h && j < n) {
        if (key_less(kx, kz, idx[j], idx[i])) tmp[k++] = idx[j++];
        else tmp[k++] = idx[i++];
    }
    while (i < h) tmp[k++] = idx[i++];
    while (j < n) tmp[k++] = idx[j++];
    memcpy(idx, tmp, (size_t)n * sizeof(int64_t));
}

/* Unique (x, z) sorted ascending (x first, then z, as unsigned), each
 * coefficient the left-to-right sum of its raw entries in input order; a term
 * is kept iff re*re + im*im > eps*eps.  Output arrays must hold m entries.
 * Returns the number of kept terms. */
int64_t orc_canonical(int64_t m, const uint64_t *x, const uint64_t *z, const double *cre,
                      const double *cim, double eps, uint64_t *ox, uint64_t *oz, double *ore,
                      double *oim)
{
    if (m <= 0) return 0;
    int64_t *idx = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) idx[i] = i;
    msort(x, z, idx, tmp, m);
    double eps2 = eps * eps;
    int64_t out = 0;
    int64_t i = 0;
    while (i < m) {
        int64_t j = i;
        double sr = 0.0, si = 0.0;
        int first = 1;
        while (j < m && x[idx[j]] == x[idx[i]] && z[idx[j]] == z[idx[i]]) {
            if (first) { sr = cre[idx[j]]; si = cim[idx[j]]; first = 0; }
            else { sr = sr + cre[idx[j]]; si = si + cim[idx[j]]; }
            ++j;
        }
        double rr = sr * sr;
        double ii = si * si;
        if (rr + ii > eps2) {
            ox[out] = x[idx[i]]; oz[out] = z[idx[i]]; ore[out] = sr; oim[out] = si;
            ++out;
        }
        i = j;
    }
    free(idx);
    free(tmp);
    return out;
}

/* ------------------------------------------------------------------------- */
/* sectors (Sec. 2.4, eq. fcidim)                                             */
/* ------------------------------------------------------------------------- */
/* A sector is either the full 2^n space (index = configuration) or a union of
 * product blocks r = (k_lo, k_hi): configurations whose low n_lo qubits hold
 * k_lo ones and whose high n - n_lo qubits hold k_hi ones.  Within a block the
 * configurations are listed in ascending numeric order (the high part varies
 * slowest); blocks follow one another in the order given. */
typedef struct {
    int n, kind, n_lo, nblk;
    int64_t dim;
    uint64_t *cfg;       /* dim configurations, index order */
    int64_t *blk_off;    /* nblk + 1 */
    int *klo, *khi;
    int32_t *inv;        /* configuration -> index, or -1 (n <= 28 only) */
    int irr;             /* 1: blocks also fix the point-group irrep of each half */
    int *irlo, *irhi;    /* irrep label of each block's low / high half */
    int qirr[64];        /* irrep label (0..7) of every qubit */
} orc_sector;

/* Irrep of a string of `bits` qubits starting at qubit `first`: the product
 * (XOR of the labels) of the irreps of its occupied orbitals (abelian point
 * group with 2^3 irreps, e.g. D2h). */
static int string_irrep(const orc_sector *s, uint64_t v, int first, int bits)
{
    int g = 0;
    for (int j = 0; j < bits; ++j)
        if ((v >> j) & 1u) g ^= s->qirr[first + j];
    return g;
}

static int64_t popc_count_list(int bits, int k, uint64_t *out)
{
    int64_t c = 0;
    uint64_t lim = ((uint64_t)1) << bits;
    for (uint64_t v = 0; v < lim; ++v)
        if (popc64(v) == k) {
            if (out) out[c] = v;
            ++c;
        }
    return c;
}

/* Number of `bits`-bit strings with k ones, by Pascal's rule
 * N(b, k) = N(b-1, k-1) + N(b-1, k), N(b, 0) = 1, N(0, k>0) = 0. */
int64_t orc_count_strings(int bits, int k)
{
    int64_t row[65];
    if (k < 0 || k > bits || bits > 64) return 0;
    for (int j = 0; j <= 64; ++j) row[j] = (j == 0) ? 1 : 0;
    for (int b = 1; b <= bits; ++b)
        for (int j = b; j >= 1; --j) row[j] = row[j] + row[j - 1];
    return row[k];
}

orc_sector *orc_sector_new(int n, int kind, int n_lo, int nblk, const int *klo, const int *khi)
{
    orc_sector *s = (orc_sector *)calloc(1, sizeof(orc_sector));
    s->n = n; s->kind = kind; s->n_lo = n_lo; s->nblk = nblk;
    s->blk_off = (int64_t *)calloc((size_t)(nblk + 1), sizeof(int64_t));
    s->klo = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    s->khi = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    if (kind == 0) {
        s->dim = ((int64_t)1) << n;
        s->cfg = (uint64_t *)malloc((size_t)s->dim * sizeof(uint64_t));
        for (int64_t i = 0; i < s->dim; ++i) s->cfg[i] = (uint64_t)i;
    } else {
        int n_hi = n - n_lo;
        int64_t total = 0;
        for (int r = 0; r < nblk; ++r) {
            s->klo[r] = klo[r];
            s->khi[r] = khi[r];
            int64_t a = popc_count_list(n_lo, klo[r], NULL);
            int64_t b = popc_count_list(n_hi, khi[r], NULL);
            s->blk_off[r] = total;
            total += a * b;
        }
        s->blk_off[nblk] = total;
        s->dim = total;
        s->cfg = (uint64_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(uint64_t));
        for (int r = 0; r < nblk; ++r) {
            int64_t a = popc_count_list(n_lo, klo[r], NULL);
            int64_t b = popc_count_list(n_hi, khi[r], NULL);
            uint64_t *lo = (uint64_t *)malloc((size_t)(a > 0 ? a : 1) * sizeof(uint64_t));
            uint64_t *hi = (uint64_t *)malloc((size_t)(b > 0 ? b : 1) * sizeof(uint64_t));
            popc_count_list(n_lo, klo[r], lo);
            popc_count_list(n_hi, khi[r], hi);
            int64_t p = s->blk_off[r];
            for (int64_t j = 0; j < b; ++j)
                for (int64_t i = 0; i < a; ++i) s->cfg[p++] = lo[i] | (hi[j] << n_lo);
            free(lo);
            free(hi);
        }
    }
    if (n <= 28) {
        int64_t full = ((int64_t)1) << n;
        s->inv = (int32_t *)malloc((size_t)full * sizeof(int32_t));
        for (int64_t v = 0; v < full; ++v) s->inv[v] = -1;
        for (int64_t i = 0; i < s->dim; ++i) s->inv[s->cfg[i]] = (int32_t)i;
    }
    return s;
}

void orc_sector_free(orc_sector *s)
{
    if (!s) return;
    free(s->cfg); free(s->blk_off); free(s->klo); free(s->khi); free(s->inv);
    free(s->irlo); free(s->irhi);
    free(s);
}

/* A sector of point-group blocks r = (k_lo, irrep_lo, k_hi, irrep_hi): the
 * configurations whose low half holds k_lo ones with irrep irrep_lo and whose
 * high half holds k_hi ones with irrep irrep_hi (qubit q has irrep
 * qubit_irrep[q]); inside a block ascending numeric order, high part slowest;
 * blocks in the order given. */
orc_sector *orc_sector_new_irrep(int n, int n_lo, int nblk, const int *klo, const int *khi, const int *irlo,
                                 const int *irhi, const int *qubit_irrep)
{
    orc_sector *s = (orc_sector *)calloc(1, sizeof(orc_sector));
    s->n = n; s->kind = 1; s->n_lo = n_lo; s->nblk = nblk; s->irr = 1;
    for (int q = 0; q < n && q < 64; ++q) s->qirr[q] = qubit_irrep[q];
    s->blk_off = (int64_t *)calloc((size_t)(nblk + 1), sizeof(int64_t));
    s->klo = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    s->khi = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    s->irlo = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    s->irhi = (int *)calloc((size_t)(nblk > 0 ? nblk : 1), sizeof(int));
    int n_hi = n - n_lo;
    uint64_t nlo = ((uint64_t)1) << n_lo, nhi = ((uint64_t)1) << n_hi;
    int64_t total = 0;
    for (int r = 0; r < nblk; ++r) {
        s->klo[r] = klo[r]; s->khi[r] = khi[r]; s->irlo[r] = irlo[r]; s->irhi[r] = irhi[r];
        int64_t a = 0, b = 0;
        for (uint64_t v = 0; v < nlo; ++v)
            if (popc64(v) == klo[r] && string_irrep(s, v, 0, n_lo) == irlo[r]) ++a;
        for (uint64_t v = 0; v < nhi; ++v)
            if (popc64(v) == khi[r] && string_irrep(s, v, n_lo, n_hi) == irhi[r]) ++b;
        s->blk_off[r] = total;
        total += a * b;
    }
    s->blk_off[nblk] = total;
    s->dim = total;
    s->cfg = (uint64_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(uint64_t));
    int64_t p = 0;
    for (int r = 0; r < nblk; ++r)
        for (uint64_t hv = 0; hv < nhi; ++hv) {
            if (popc64(hv) != khi[r] || string_irrep(s, hv, n_lo, n_hi) != irhi[r]) continue;
            for (uint64_t lv = 0; lv < nlo; ++lv)
                if (popc64(lv) == klo[r] && string_irrep(s, lv, 0, n_lo) == irlo[r]) s->cfg[p++] = lv | (hv << n_lo);
        }
    if (n <= 28) {
        int64_t full = ((int64_t)1) << n;
        s->inv = (int32_t *)malloc((size_t)full * sizeof(int32_t));
        for (int64_t v = 0; v < full; ++v) s->inv[v] = -1;
        for (int64_t i = 0; i < s->dim; ++i) s->inv[s->cfg[i]] = (int32_t)i;
    }
    return s;
}

int64_t orc_sector_dim(const orc_sector *s) { return s->dim; }

void orc_sector_configs(const orc_sector *s, uint64_t *out)
{
    memcpy(out, s->cfg, (size_t)s->dim * sizeof(uint64_t));
}

/* Index of configuration b, or -1 if b is not in the sector: the position of
 * b in the enumeration (table lookup for n <= 28, otherwise a binary search in
 * the sorted list of the block that b's popcounts select). */
int64_t orc_sector_index(const orc_sector *s, uint64_t b)
{
    if (s->n < 64 && (b >> s->n) != 0) return -1;
    if (s->inv) return (int64_t)s->inv[b];
    if (s->kind == 0) return (int64_t)b;
    uint64_t lomask = (s->n_lo == 0) ? 0 : ((((uint64_t)1) << s->n_lo) - 1);
    int kl = popc64(b & lomask), kh = popc64(b >> s->n_lo);
    for (int r = 0; r < s->nblk; ++r) {
        if (s->klo[r] != kl || s->khi[r] != kh) continue;
        if (s->irr && (string_irrep(s, b & lomask, 0, s->n_lo) != s->irlo[r] ||
                       string_irrep(s, b >> s->n_lo, s->n_lo, s->n - s->n_lo) != s->irhi[r]))
            continue;
        int64_t lo = s->blk_off[r], hi = s->blk_off[r + 1] - 1;
        while (lo <= hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (s->cfg[mid] == b) return mid;
            if (s->cfg[mid] < b) lo = mid + 1;
            else hi = mid - 1;
        }
        return -1;
    }
    return -1;
}

void orc_sector_rank_many(const orc_sector *s, int64_t cnt, const uint64_t *b, int64_t *idx)
{
    for (int64_t i = 0; i < cnt; ++i) idx[i] = orc_sector_index(s, b[i]);
}

/* ------------------------------------------------------------------------- */
/* operator-state products                                                   */
/* ------------------------------------------------------------------------- */
static int parity(uint64_t v) { return popc64(v) & 1; }

/* out = P_S H P_S psi, source form of eq. grouped_contraction, term by term:
 * for every term k and source s in the sector, t = s XOR X_k; if t is in the
 * sector, out[t] += C_k (-1)^popc(Z_k & s) psi[s].  psi, out: interleaved
 * (re, im) doubles of length 2*dim. */
void orc_apply(const orc_sector *s, int64_t m, const uint64_t *x, const uint64_t *z,
               const double *cre, const double *cim, const double *psi, double *out)
{
    int64_t D = s->dim;
    for (int64_t i = 0; i < 2 * D; ++i) out[i] = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        cplx C = c_make(cre[k], cim[k]);
        for (int64_t si = 0; si < D; ++si) {
            uint64_t b = s->cfg[si];
            int64_t ti = orc_sector_index(s, b ^ x[k]);
            if (ti < 0) continue;
            cplx a = c_mul(C, c_make(psi[2 * si], psi[2 * si + 1]));
            if (parity(z[k] & b)) a = c_make(-a.re, -a.im);
            cplx o = c_add(c_make(out[2 * ti], out[2 * ti + 1]), a);
            out[2 * ti] = o.re;
            out[2 * ti + 1] = o.im;
        }
    }
}

/* Selected rows of P_S H P_S psi by the matrix-element definition
 * (H psi)_t = sum_k C_k <t|P_k|psi> = sum_k C_k (-1)^popc(Z_k & s) psi[s],
 * s = t XOR X_k, for target indices tidx[0..nt). */
void orc_apply_rows(const orc_sector *s, int64_t m, const uint64_t *x, const uint64_t *z,
                    const double *cre, const double *cim, const double *psi, int64_t nt,
                    const int64_t *tidx, double *out)
{
    for (int64_t j = 0; j < nt; ++j) {
        uint64_t t = s->cfg[tidx[j]];
        cplx acc = c_make(0.0, 0.0);
        for (int64_t k = 0; k < m; ++k) {
            uint64_t b = t ^ x[k];
            int64_t si = orc_sector_index(s, b);
            if (si < 0) continue;
            cplx a = c_mul(c_make(cre[k], cim[k]), c_make(psi[2 * si], psi[2 * si + 1]));
            if (parity(z[k] & b)) a = c_make(-a.re, -a.im);
            acc = c_add(acc, a);
        }
        out[2 * j] = acc.re;
        out[2 * j + 1] = acc.im;
    }
}

/* eq. vqe_energy: E = <psi|H|psi> = sum_t conj(psi_t) (H psi)_t, and the
 * squared norm <H psi|H psi>, both as plain sequential FP64 sums.
 * res = {Re E, Im E, ||H psi||^2}. */
void orc_expect(const orc_sector *s, int64_t m, const uint64_t *x, const uint64_t *z,
                const double *cre, const double *cim, const double *psi, double *res)
{
    int64_t D = s->dim;
    double *hp = (double *)malloc((size_t)(2 * D > 0 ? 2 * D : 1) * sizeof(double));
    orc_apply(s, m, x, z, cre, cim, psi, hp);
    double er = 0.0, ei = 0.0, n2 = 0.0;
    for (int64_t t = 0; t < D; ++t) {
        cplx c = c_mul(c_make(psi[2 * t], -psi[2 * t + 1]), c_make(hp[2 * t], hp[2 * t + 1]));
        er += c.re;
        ei += c.im;
        n2 += hp[2 * t] * hp[2 * t] + hp[2 * t + 1] * hp[2 * t + 1];
    }
    res[0] = er;
    res[1] = ei;
    res[2] = n2;
    free(hp);
}

/* Does G take some sector configuration out of the sector?  For each sector
 * configuration b and each target t = b XOR X_k outside the sector, sum the
 * coefficients of G|b> at t; any nonzero sum is a leak.  Returns 1 on a leak. */
int orc_leaks(const orc_sector *s, int64_t m, const uint64_t *x, const uint64_t *z,
              const double *cre, const double *cim)
{
    for (int64_t si = 0; si < s->dim; ++si) {
        uint64_t b = s->cfg[si];
        for (int64_t k = 0; k < m; ++k) {
            uint64_t t = b ^ x[k];
            if (orc_sector_index(s, t) >= 0) continue;
            cplx acc = c_make(0.0, 0.0);
            for (int64_t j = 0; j < m; ++j) {
                if ((b ^ x[j]) != t) continue;
                cplx a = c_make(cre[j], cim[j]);
                if (parity(z[j] & b)) a = c_make(-a.re, -a.im);
                acc = c_add(acc, a);
            }
            if (acc.re != 0.0 || acc.im != 0.0) return 1;
        }
    }
    return 0;
}

/* psi <- exp(-i theta G) psi by the Taylor series sum_j (-i theta G)^j / j!,
 * each power applied with orc_apply.  The angle is split into nsub equal
 * pieces with |theta/nsub| * sum_k |C_k| <= 1/2 and each piece summed until a
 * term's norm falls below 1e-18 of the state's.  psi: interleaved, in place. */
void orc_rotate(const orc_sector *s, int64_t m, const uint64_t *x, const uint64_t *z,
                const double *cre, const double *cim, double theta, double *psi)
{
    int64_t D = s->dim;
    double bound = 0.0;
    for (int64_t k = 0; k < m; ++k) bound += sqrt(cre[k] * cre[k] + cim[k] * cim[k]);
    int nsub = (int)ceil(fabs(theta) * bound / 0.5);
    if (nsub < 1) nsub = 1;
    double th = theta / nsub;
    double *term = (double *)malloc((size_t)(2 * D > 0 ? 2 * D : 1) * sizeof(double));
    double *nxt = (double *)malloc((size_t)(2 * D > 0 ? 2 * D : 1) * sizeof(double));
    double *acc = (double *)malloc((size_t)(2 * D > 0 ? 2 * D : 1) * sizeof(double));
    for (int sub = 0; sub < nsub; ++sub) {
        double nrm = 0.0;
        for (int64_t i = 0; i < 2 * D; ++i) {
            term[i] = psi[i];
            acc[i] = psi[i];
            nrm += psi[i] * psi[i];
        }
        for (int j = 1; j < 200; ++j) {
            orc_apply(s, m, x, z, cre, cim, term, nxt);
            /* term <- (-i th / j) * (G term) */
            double tn = 0.0;
            for (int64_t t = 0; t < D; ++t) {
                cplx v = c_make(nxt[2 * t], nxt[2 * t + 1]);
                v = c_mul(v, c_make(0.0, -th / (double)j));
                term[2 * t] = v.re;
                term[2 * t + 1] = v.im;
                acc[2 * t] += v.re;
                acc[2 * t + 1] += v.im;
                tn += v.re * v.re + v.im * v.im;
            }
            if (tn <= 1e-36 * nrm) break;
        }
        for (int64_t i = 0; i < 2 * D; ++i) psi[i] = acc[i];
    }
    free(term);
    free(nxt);
    free(acc);
}

/* ------------------------------------------------------------------------- */
/* Hartree-Fock energy (Slater-Condon closed form)                           */
/* ------------------------------------------------------------------------- */
/* Determinant with alpha orbitals 0..na-1 and beta orbitals 0..nb-1 occupied:
 *   E = sum_sigma sum_{i occ} h_ii
 *     + 1/2 sum_{sigma, tau} sum_{i in sigma, j in tau} (ii|jj)
 *     - 1/2 sum_sigma sum_{i, j in sigma} (ij|ji)  + e_nn.                    */
double orc_hf_energy(int norb, const double *h, const double *g, int na, int nb, double e_nn)
{
    int nocc[2] = {na, nb};
    double e = 0.0;
    for (int sg = 0; sg < 2; ++sg)
        for (int i = 0; i < nocc[sg]; ++i) e += h[i * norb + i];
    double j = 0.0, k = 0.0;
    for (int sg = 0; sg < 2; ++sg)
        for (int tu = 0; tu < 2; ++tu)
            for (int i = 0; i < nocc[sg]; ++i)
                for (int jj = 0; jj < nocc[tu]; ++jj) {
                    j += g[((i * norb + i) * norb + jj) * norb + jj];
                    if (sg == tu) k += g[((i * norb + jj) * norb + jj) * norb + i];
                }
    return e + 0.5 * j - 0.5 * k + e_nn;
}
