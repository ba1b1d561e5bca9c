"""Writes the stored expected values under tests/golden/ by calling only the oracle.

    python tests/golden/make_golden.py

p3_dense_k.json: infinite-crystal (k-integrated dense diagonalisation, 8^3 Bloch phases)
rho, mu, energies and paper-form stress of a 4^3-node periodic cell with two atoms; the
infinite-cell SQ oracle must converge to these as R_cut and n_pl grow (Sec. 4: the
infinite-cell method gives the infinite-crystal result without Brillouin-zone integration).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense_k  # noqa: E402
from oracle.sq_oracle import Problem  # noqa: E402
from workloads import tiny_instance  # noqa: E402

P3_CASE = dict(seed=1, n=[4, 4, 4], h=[0.9, 0.9, 0.9], n_o=2, kT=3.17,
               pos=[[0.7, 1.3, 2.2], [2.5, 2.9, 0.4]], n_e=2, r_cut=1.8, n_pl=20)
P3_NK = 8


def p3():
    prob = Problem(tiny_instance(**P3_CASE))
    o = dense_k.observables(prob, nk=P3_NK)
    return {
        "case": P3_CASE, "nk": P3_NK,
        "mu": o["mu"], "E_band": o["E_band"], "E_s": o["E_s"], "E_nl": o["E_nl"],
        "rho": o["rho"].tolist(), "sigma": o["sigma"].tolist(),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "p3_dense_k.json"), "w") as f:
        json.dump(p3(), f, indent=1)
    print("wrote p3_dense_k.json")
