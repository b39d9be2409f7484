"""Oracle of the multi-word-mask operator algebra (more than 64 qubits).

TEST INFRASTRUCTURE ONLY (imported by tests/).

Strings are Python integers (bit q of x / z = qubit q, any width).  The
definitions are those of oracle.c written for unbounded masks:
* a letter string is multiplied qubit by qubit with the textbook table
  (XY = iZ, YZ = iX, ZX = iY, reversed order -i; oracle.letter_mul);
* the XZ-form coefficient of a letter string with coefficient c is
  C = c i^popcount(x & z) (Sec. 2.2.2);
* a_P = 1/2 (X_P + i Y_P) Z_{<P}, a_P^dagger = 1/2 (X_P - i Y_P) Z_{<P} as
  letter sums [X version, Y version], products of ladder operators expanded
  term by term with the left factor most significant (the raw order);
* canonical form: equal (x, z) summed left to right in raw order, terms with
  re^2 + im^2 <= eps^2 dropped, (x, z) ascending (x first).
Pinned in tests/test_oracle_wide.py: identical to the 64-bit C oracle on
strings of at most 64 qubits, and the canonical anticommutators
{a_P, a_Q^dagger} = delta_PQ for modes above 64.
"""
from __future__ import annotations

from . import letter_mul

_I = [1, 1j, -1, -1j]


# letter codes of oracle.letter_mul: I = 0, X = 1, Y = 2, Z = 3
def _letter(x, z, q):
    """Letter at qubit q of the string with bits (x, z): (0,0) I, (1,0) X, (0,1) Z, (1,1) Y."""
    return [0, 1, 3, 2][((x >> q) & 1) | (((z >> q) & 1) << 1)]
def _bits(letter):
    return {0: (0, 0), 1: (1, 0), 2: (1, 1), 3: (0, 1)}[letter]


def string_mul(n, xa, za, xb, zb):
    """Letter-string product: (x, z, k) with phase i^k."""
    x = z = 0
    k = 0
    for q in range(n):
        u = _letter(xa, za, q)
        v = _letter(xb, zb, q)
        if u == 0 and v == 0:
            continue
        w, kk = letter_mul(u, v)
        k += kk
        bx, bz = _bits(w)
        x |= bx << q
        z |= bz << q
    return x, z, k % 4


def popcount(v):
    return bin(v).count("1")


def ladder(P, dagger):
    """[(x, z, c_letter)]: X version then Y version of a_P (or a_P^dagger)."""
    below = (1 << P) - 1
    ysign = -1j if dagger else 1j
    return [(1 << P, below, 0.5), (1 << P, below | (1 << P), 0.5 * ysign)]


def canonical(entries, eps=0.0):
    """entries: [(x, z, C)] in raw order -> sorted [(x, z, C)]."""
    acc = {}
    for x, z, c in entries:
        key = (x, z)
        acc[key] = acc[key] + c if key in acc else c
    out = [(x, z, c) for (x, z), c in acc.items() if c.real * c.real + c.imag * c.imag > eps * eps]
    out.sort(key=lambda t: (t[0], t[1]))
    return out


def fermion_sum(n, terms, eps=0.0):
    """Canonical XZ-form sum of sum_t c_t prod_j f_{t,j}; terms = [(c, [(mode, dagger), ...])]."""
    raw = []
    for c, factors in terms:
        strings = [(0, 0, complex(c))]
        for P, dag in factors:
            lad = ladder(P, dag)
            nxt = []
            for xa, za, ca in strings:          # left factors outer
                for xb, zb, cb in lad:          # [X version, Y version]
                    x, z, k = string_mul(n, xa, za, xb, zb)
                    nxt.append((x, z, ca * cb * _I[k]))
            strings = nxt
        for x, z, cl in strings:
            raw.append((x, z, cl * _I[popcount(x & z) % 4]))
    return canonical(raw, eps)


def product(n, A, B, eps=0.0):
    """Canonical A B of two canonical XZ-form sums (pairs a-major)."""
    raw = []
    for xa, za, ca in A:
        la = ca * _I[(4 - popcount(xa & za) % 4) % 4]
        for xb, zb, cb in B:
            lb = cb * _I[(4 - popcount(xb & zb) % 4) % 4]
            x, z, k = string_mul(n, xa, za, xb, zb)
            raw.append((x, z, (la * lb) * _I[(k + popcount(x & z)) % 4]))
    return canonical(raw, eps)


def add(A, B, beta=1.0, eps=0.0):
    return canonical(list(A) + [(x, z, beta * c) for x, z, c in B], eps)
