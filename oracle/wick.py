"""Brute-force Wick enumeration of the nucleon two-point function (test infrastructure only).

Instead of the two printed contractions, this routine starts from the
interpolating fields of Sec. 4,
    N_alpha     = eps^{abc} (u^{aT} C g5 d^b) d^c_alpha,
    Nbar_beta   = eps^{feg} dbar^e_beta (dbar^f C g5 ubar^{gT}),
writes <N_alpha Nbar_beta> as a product of six Grassmann fields, enumerates
every complete pairing of a quark with an antiquark of the same flavour,
computes the sign of each pairing from the parity of the permutation that
brings every pair next to each other, and evaluates the resulting sums with
einsum.  C_N(y0) = sum_{y vec} sum_{alpha beta} <N_alpha Nbar_beta> (P-)_{beta alpha}
with <q(y) qbar(x)> = S(y,x) for u and d alike.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import gamma as _gamma


def _perm_parity(perm):
    perm = list(perm)
    sign = 1
    for i in range(len(perm)):
        while perm[i] != i:
            j = perm[i]
            perm[i], perm[j] = perm[j], perm[i]
            sign = -sign
    return sign


def levi_civita():
    e = np.zeros((3, 3, 3))
    for p in itertools.permutations(range(3)):
        e[p] = _perm_parity(p)
    return e


# The field string of N_alpha(y) Nbar_beta(x): (flavour, is_bar, spin label, colour label)
_FIELDS = [
    ("u", False, "r", "a"),   # u^a_rho
    ("d", False, "s", "b"),   # d^b_sigma
    ("d", False, "A", "c"),   # d^c_alpha
    ("d", True, "B", "e"),    # dbar^e_beta
    ("d", True, "k", "f"),    # dbar^f_kappa
    ("u", True, "l", "g"),    # ubar^g_lambda
]


def pairings():
    """All complete pairings as (sign, [(quark_pos, antiquark_pos), ...])."""
    quarks = [i for i, f in enumerate(_FIELDS) if not f[1]]
    antis = [i for i, f in enumerate(_FIELDS) if f[1]]
    out = []
    for perm in itertools.permutations(antis):
        if any(_FIELDS[q][0] != _FIELDS[a][0] for q, a in zip(quarks, perm)):
            continue
        order = []
        for q, a in zip(quarks, perm):
            order += [q, a]
        out.append((_perm_parity(order), list(zip(quarks, perm))))
    return out


def nucleon_correlator(S_sites, y0_of_site, T):
    """S_sites: (n, 4, 3, 4, 3) = S(y,x)_{rho a, sigma b} per sink site.
    Returns C_N(y0) for y0 in range(T) (complex)."""
    g = _gamma()
    C = 1j * g[0] @ g[2]
    Cg5 = C @ g[4]
    Pm = 0.5 * (np.eye(4) - g[0])
    eps = levi_civita()
    per_site = np.zeros(S_sites.shape[0], dtype=np.complex128)
    for sign, pairs in pairings():
        # operands: eps_abc, eps_feg, Cg5_{r s}, Cg5_{k l}, Pm_{B A}, then one S per pair
        terms = ["abc", "feg", "rs", "kl", "BA"]
        ops = [eps, eps, Cg5, Cg5, Pm]
        for q, a in pairs:
            terms.append("n" + _FIELDS[q][2] + _FIELDS[q][3] + _FIELDS[a][2] + _FIELDS[a][3])
            ops.append(S_sites)
        expr = ",".join(terms) + "->n"
        per_site += sign * np.einsum(expr, *ops, optimize=True)
    out = np.zeros(T, dtype=np.complex128)
    np.add.at(out, y0_of_site, per_site)
    return out
