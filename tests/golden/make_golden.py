"""Writes the golden free-field values used by tests/test_oracle.py.

Only the oracle's closed forms are called (oracle/freefield.py, oracle/wick.py):
with unit links the Wilson propagator of App. A is diagonal in momentum space,
S(y,0) = (1/V) sum_p e^{ipy} D(p)^{-1}, and the pion (Eq. W0pc with the exact S)
and nucleon (Sec. 4) correlators follow from it.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import freefield, wick  # noqa: E402


def main():
    L = (8, 4, 4, 4)
    kappa = 0.12
    S = freefield.momentum_propagator(L, kappa, 1).reshape(-1, 4, 4)   # antiperiodic in time
    V = S.shape[0]
    vol3 = L[1] * L[2] * L[3]
    y0 = np.arange(V) // vol3
    pion = np.zeros(L[0])
    np.add.at(pion, y0, 3 * np.sum(np.abs(S) ** 2, axis=(1, 2)))      # colour identity: 3 copies
    blocks = np.einsum("yrs,ab->yrasb", S, np.eye(3))
    nucleon = wick.nucleon_correlator(blocks, y0, L[0])
    out = {
        "description": "free Wilson quark (unit links), 8x4^3, antiperiodic time, kappa 0.12, point source at the "
                       "origin: pion sum_y tr S S^+ per time slice and nucleon sum_y (W_N1 - W_N2) per time slice",
        "source": "closed form in momentum space of the App. A operator; correlators of Sec. 4 (Eq. W0pc, nucleon)",
        "lattice": list(L), "kappa": kappa, "time_bc": "antiperiodic",
        "pion": pion.tolist(),
        "nucleon_re": nucleon.real.tolist(), "nucleon_im": nucleon.imag.tolist(),
    }
    with open(os.path.join(HERE, "free_field_8x4x4x4.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
