"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws random numbers and lays them out as plain arrays.  It holds
none of the method's arithmetic: no Pauli products, no Jordan--Wigner mapping,
no sector ranking, no operator application.  Each side (``oracle/`` and the CUDA
library) turns these arrays into Pauli sums and results on its own.

The paper's own benchmarks use PySCF integrals of real molecules (Sec. 3.2,
Table 2), which are not available here; the generators below stand in for them
with integrals of the same shape and symmetry (a symmetric one-body matrix and
an 8-fold-symmetric two-body tensor in chemist notation, as in Sec. 3.1.1).

All draws use numpy's ``default_rng`` (PCG64) with the seeds stated per workload.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Letter encoding of a single-qubit Pauli operator as the bit pair (a, b) of
# Sec. 2.2.1: I=(0,0), X=(1,0), Y=(1,1), Z=(0,1).  A string is the pair of masks
# (x, z) with bit k of x = a_k and bit k of z = b_k.
LETTER_FORM = 0  # coefficient multiplies the letter string (Y is a letter)
XZ_FORM = 1      # coefficient multiplies X^x Z^z (the symplectic form)


# ----------------------------------------------------------------------------
# molecular integrals
# ----------------------------------------------------------------------------
def draw_h(rng: np.random.Generator, norb: int) -> np.ndarray:
    """One-body integrals: h_pq = N(0,1) * exp(-|p-q|/2), symmetric.

    Draw order: for p ascending, for q >= p ascending.
    """
    h = np.zeros((norb, norb), dtype=np.float64)
    for p in range(norb):
        for q in range(p, norb):
            v = rng.normal(0.0, 1.0) * math.exp(-abs(p - q) / 2.0)
            h[p, q] = v
            h[q, p] = v
    return h


def draw_g(rng: np.random.Generator, norb: int) -> np.ndarray:
    """Two-body integrals (pq|rs) in chemist notation with 8-fold symmetry.

    v = N(0, sd=0.1) * exp(-(|p-q| + |r-s|)/3), drawn once per unique
    (pq, rs) pair index (pq = p(p+1)/2 + q with q <= p, same for rs, pq >= rs),
    loops p, q, r, s ascending, and written to all 8 images.
    """
    g = np.zeros((norb, norb, norb, norb), dtype=np.float64)
    for p in range(norb):
        for q in range(p + 1):
            pq = p * (p + 1) // 2 + q
            for r in range(norb):
                for s in range(r + 1):
                    rs = r * (r + 1) // 2 + s
                    if pq < rs:
                        continue
                    v = rng.normal(0.0, 0.1) * math.exp(-(abs(p - q) + abs(r - s)) / 3.0)
                    for (a, b, c, d) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
                        g[a, b, c, d] = v
    return g


def molecular_integrals(norb: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(h, g) for a synthetic molecule with ``norb`` spatial orbitals."""
    rng = np.random.default_rng(seed)
    h = draw_h(rng, norb)
    g = draw_g(rng, norb)
    return h, g


def pes_integrals(norb: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(h0, h1, g0) for the potential-energy scan h(R) = h0 + R h1, g(R) = g0 exp(-0.3 R).

    Drawn from one stream: h0, then g0, then h1.
    """
    rng = np.random.default_rng(seed)
    h0 = draw_h(rng, norb)
    g0 = draw_g(rng, norb)
    h1 = draw_h(rng, norb)
    return h0, h1, g0


def pes_point(h0, h1, g0, R: float) -> tuple[np.ndarray, np.ndarray]:
    return h0 + R * h1, g0 * math.exp(-0.3 * R)


# ----------------------------------------------------------------------------
# spin chain (letter-form Pauli terms: the problem is *given* as a Pauli sum)
# ----------------------------------------------------------------------------
def xxz_couplings(n_sites: int, seed: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """J_xy ~ U[0.5,1.5], J_z ~ U[-1,1] per bond, h_z ~ N(0, sd=0.5) per site."""
    rng = np.random.default_rng(seed)
    jxy = rng.uniform(0.5, 1.5, n_sites - 1)
    jz = rng.uniform(-1.0, 1.0, n_sites - 1)
    hz = rng.normal(0.0, 0.5, n_sites)
    return jxy, jz, hz


def xxz_terms(n_sites: int, seed: int):
    """Open XXZ chain H = sum_i Jxy_i (X_i X_i+1 + Y_i Y_i+1) + Jz_i Z_i Z_i+1 + sum_i h_i Z_i.

    Returned as letter-form arrays (x, z, c_re, c_im): a letter string has
    qubit k = X if only x has bit k, Y if both, Z if only z.
    """
    jxy, jz, hz = xxz_couplings(n_sites, seed)
    xs, zs, cs = [], [], []
    for i in range(n_sites - 1):
        b = (1 << i) | (1 << (i + 1))
        xs.append(b); zs.append(0); cs.append(jxy[i])   # X X
        xs.append(b); zs.append(b); cs.append(jxy[i])   # Y Y
        xs.append(0); zs.append(b); cs.append(jz[i])    # Z Z
    for i in range(n_sites):
        xs.append(0); zs.append(1 << i); cs.append(hz[i])  # Z
    x = np.array(xs, dtype=np.uint64)
    z = np.array(zs, dtype=np.uint64)
    c = np.array(cs, dtype=np.float64)
    return x, z, c, np.zeros_like(c)


def tfim_terms(n_sites: int, J: float = 0.25, h: float = 1.0):
    """Open transverse-field Ising chain of Sec. 3.5, letter form."""
    xs, zs, cs = [], [], []
    for i in range(n_sites - 1):
        xs.append(0); zs.append((1 << i) | (1 << (i + 1))); cs.append(J)
    for i in range(n_sites):
        xs.append(1 << i); zs.append(0); cs.append(h)
    c = np.array(cs, dtype=np.float64)
    return np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64), c, np.zeros_like(c)


def neel_config(n_sites: int) -> int:
    """Neel basis configuration: bit i set for odd i."""
    return sum(1 << i for i in range(1, n_sites, 2))


def random_masks(rng: np.random.Generator, n: int, m: int) -> np.ndarray:
    """m uniformly random n-bit masks (n <= 64) as uint64."""
    lo = rng.integers(0, 1 << 32, m, dtype=np.uint64)
    hi = rng.integers(0, 1 << 32, m, dtype=np.uint64)
    v = lo | (hi << np.uint64(32))
    if n < 64:
        v &= np.uint64((1 << n) - 1)
    return v


def random_pauli_terms(n: int, m: int, seed: int, dup_frac: float = 0.3):
    """Random terms (x, z, gamma, c_re, c_im) with some repeated strings (merge tests)."""
    rng = np.random.default_rng(seed)
    x = random_masks(rng, n, m)
    z = random_masks(rng, n, m)
    ndup = int(dup_frac * m)
    if ndup and m > 1:
        src = rng.integers(0, m, ndup)
        dst = rng.integers(0, m, ndup)
        x[dst] = x[src]
        z[dst] = z[src]
    gamma = rng.integers(0, 4, m).astype(np.uint8)
    cre = rng.normal(size=m)
    cim = rng.normal(size=m)
    return x, z, gamma, cre, cim


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------
def random_state(dim: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """re, im ~ N(0,1) from default_rng(seed), normalised to unit 2-norm."""
    rng = np.random.default_rng(seed)
    re = rng.normal(size=dim)
    im = rng.normal(size=dim)
    v = (re + 1j * im).astype(np.complex128)
    v /= np.linalg.norm(v)
    return v.astype(dtype)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
@dataclass
class Molecular:
    norb: int
    n_alpha: int
    n_beta: int
    seed: int
    psi_seed: int

    @property
    def n_qubits(self) -> int:
        return 2 * self.norb

    @property
    def dim(self) -> int:
        return math.comb(self.norb, self.n_alpha) * math.comb(self.norb, self.n_beta)

    def integrals(self):
        return molecular_integrals(self.norb, self.seed)


# 12 qubits, 6 spatial orbitals, (3a,3b) sector of dim 400, seed 0
MOL12 = Molecular(norb=6, n_alpha=3, n_beta=3, seed=0, psi_seed=11)
# 24 qubits, 12 spatial orbitals, (6a,6b) sector of dim 853,776, seed 0
MOL24 = Molecular(norb=12, n_alpha=6, n_beta=6, seed=0, psi_seed=12)


def batched_states(n_states: int = 64, seed: int = 3):
    """64 independent molecules: norb ~ U{8..14}, half filling Na = Nb = floor(norb/2).

    Integrals for state b use seed 1000+b, its state vector seed 2000+b.
    """
    rng = np.random.default_rng(seed)
    norbs = rng.integers(8, 15, n_states)
    out = []
    for b, no in enumerate(norbs):
        no = int(no)
        out.append(Molecular(norb=no, n_alpha=no // 2, n_beta=no // 2, seed=1000 + b, psi_seed=2000 + b))
    return out


XXZ_SITES = 30
XXZ_SEED = 1
PES_NORB = 16
PES_SEED = 2
PES_POINTS = [0.5 + 2.5 * i / 39 for i in range(40)]


# ----------------------------------------------------------------------------
# excitation generators, described as fermionic monomials (mode, dagger) lists
# ----------------------------------------------------------------------------
def pair_double_generator(norb: int, p: int, q: int):
    """G = i (T - T^dagger), T = a+_{q,alpha} a+_{q,beta} a_{p,beta} a_{p,alpha}.

    G is Hermitian, so exp(-i theta G) = exp(theta tau) with the anti-Hermitian
    tau = T - T^dagger of the paper's Trotter factors (Sec. 3.2).  Spin orbital
    of (orbital r, alpha) is r, of (r, beta) is norb + r.
    """
    qa, qb, pa, pb = q, norb + q, p, norb + p
    return [(1j, [(qa, 1), (qb, 1), (pb, 0), (pa, 0)]),
            (-1j, [(pa, 1), (pb, 1), (qb, 0), (qa, 0)])]


def single_generator(norb: int, p: int, q: int, spin: int):
    """G = i (a+_q a_p - a+_p a_q) for one spin (0 alpha, 1 beta)."""
    P, Q = spin * norb + p, spin * norb + q
    return [(1j, [(Q, 1), (P, 0)]), (-1j, [(P, 1), (Q, 0)])]


def pair_double_ansatz(norb: int, count: int):
    """Generalized pair doubles (p < q, lexicographic), repeated in layers and
    truncated to `count` generators."""
    base = [(p, q) for p in range(norb) for q in range(p + 1, norb)]
    out = []
    while len(out) < count:
        out.extend(base)
    return out[:count]


def seniority_zero_configs(norb: int, npairs: int) -> np.ndarray:
    """Every configuration whose beta string equals its alpha string (alpha in
    the low norb bits, beta in the high ones), npairs electrons of each spin,
    ascending: the configurations a pair-double ansatz reaches from a
    closed-shell reference.  C(norb, npairs) entries (uint64)."""
    out = [a | (a << norb) for a in range(1 << norb) if bin(a).count("1") == npairs]
    return np.array(sorted(out), dtype=np.uint64)


def double_generator(modes_c, modes_a):
    """G = i (T - T^dagger), T = a+_{c0} a+_{c1} a_{a1} a_{a0} (creation modes c,
    annihilation modes a, spin-orbital indices)."""
    c0, c1 = modes_c
    a0, a1 = modes_a
    return [(1j, [(c0, 1), (c1, 1), (a1, 0), (a0, 0)]),
            (-1j, [(a0, 1), (a1, 1), (c1, 0), (c0, 0)])]


def uccsd_pool(norb: int, na: int, nb: int, generalized: bool = False):
    """Spin-conserving single and double excitation generators G = i (T - T^dagger)
    of a UCCSD (or, generalized=True, UCCGSD) ansatz in blocked spin order
    (alpha orbital r = mode r, beta orbital r = mode norb + r).

    UCCSD: occupied = the lowest na alpha / nb beta orbitals, excitations from
    occupied to virtual.  UCCGSD: every ordered pair of distinct orbital sets.
    Order: alpha singles, beta singles, alpha-alpha doubles, beta-beta doubles,
    alpha-beta doubles; each list lexicographic.  Returns [(label, terms)]."""
    occ = {0: list(range(na)), 1: list(range(nb))}
    vir = {0: list(range(na, norb)), 1: list(range(nb, norb))}
    out = []
    for spin in (0, 1):
        src = range(norb) if generalized else occ[spin]
        for p in src:
            for q in (range(p + 1, norb) if generalized else vir[spin]):
                out.append((f"s{'ab'[spin]}_{p}_{q}", single_generator(norb, p, q, spin)))
    for spin in (0, 1):
        base = spin * norb
        if generalized:
            pairs = [(p, q) for p in range(norb) for q in range(p + 1, norb)]
            combos = [(a, b) for i, a in enumerate(pairs) for b in pairs[i + 1:]]
        else:
            op = [(i, j) for i in occ[spin] for j in occ[spin] if i < j]
            vp = [(a, b) for a in vir[spin] for b in vir[spin] if a < b]
            combos = [(o, v) for o in op for v in vp]
        for (i, j), (a, b) in combos:
            out.append((f"d{'ab'[spin]}{'ab'[spin]}_{i}{j}_{a}{b}",
                        double_generator((base + a, base + b), (base + i, base + j))))
    if generalized:
        ab = [((i, j), (a, b)) for i in range(norb) for j in range(norb) for a in range(norb) for b in range(norb)
              if (i, j) < (a, b)]
    else:
        ab = [((i, j), (a, b)) for i in occ[0] for j in occ[1] for a in vir[0] for b in vir[1]]
    for (i, j), (a, b) in ab:
        out.append((f"dab_{i}{j}_{a}{b}", double_generator((a, norb + b), (i, norb + j))))
    return out


def uccsd_trotter_order(pool, norb: int):
    """One Trotter step's factor order for a UCCSD / UCCGSD pool: the alpha-only
    generators (singles, then doubles), the beta-only ones, then the alpha-beta
    doubles grouped by their beta excitation (the pool's labels give the spin
    cases; a product formula may take its factors in any fixed order)."""
    def key(item):
        label, terms = item
        kind = label.split("_")[0]
        if kind in ("sa", "daa"):
            return (0, 0)
        if kind in ("sb", "dbb"):
            return (1, 0)
        modes = sorted({m for m, _ in terms[0][1] if m >= norb})
        return (2, tuple(modes))
    return sorted(pool, key=key)  # stable: the pool's order inside each class


# ----------------------------------------------------------------------------
# abelian point-group symmetry (synthetic irrep labels)
# ----------------------------------------------------------------------------
def orbital_irreps(norb: int, seed: int = 4000, n_irreps: int = 8) -> np.ndarray:
    """Seeded irrep label (0..n_irreps-1, an abelian group of order 8 such as
    D2h, product = XOR) of every spatial orbital."""
    return np.random.default_rng(seed).integers(0, n_irreps, norb).astype(np.int32)


def pointgroup_integrals(norb: int, seed: int, irreps) -> tuple[np.ndarray, np.ndarray]:
    """The molecular generator's integrals with the entries that the point group
    forbids set to zero: h_pq unless irrep(p) = irrep(q), (pq|rs) unless
    irrep(p) ^ irrep(q) ^ irrep(r) ^ irrep(s) = 0."""
    h, g = molecular_integrals(norb, seed)
    ir = np.asarray(irreps)
    h = np.where(ir[:, None] == ir[None, :], h, 0.0)
    sym = (ir[:, None, None, None] ^ ir[None, :, None, None] ^ ir[None, None, :, None] ^ ir[None, None, None, :]) == 0
    g = np.where(sym, g, 0.0)
    return h, g


def pointgroup_blocks(norb: int, na: int, nb: int, total_irrep: int, irreps):
    """The nonempty blocks (k_lo, irrep_lo, k_hi, irrep_hi) of the sector with na
    alpha and nb beta electrons and total irrep `total_irrep`, alpha irrep
    ascending (blocked spin order: alpha = low half)."""
    from itertools import combinations
    ir = [int(v) for v in irreps]
    def present(k):
        out = set()
        for c in combinations(range(norb), k):
            g = 0
            for p in c:
                g ^= ir[p]
            out.add(g)
        return out
    pa, pb = present(na), present(nb)
    return [(na, ga, nb, ga ^ total_irrep) for ga in range(8) if ga in pa and (ga ^ total_irrep) in pb]
