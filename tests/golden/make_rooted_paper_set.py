"""Writes rooted_paper_set.json: the oracle's trajectory for the parameter set
of the paper's rooted kappa^4 run (Sec. IV.B: kappa^4 Mtilde, root N = 8,
polynomials of degrees n_1 = 16 and n_2 = 42, remainder force truncated at
n_t = 160, leapfrog on four Sexton-Weingarten levels with m_0 = 40, m_1 = 3,
m_2 = 2 and m = 4 outer steps, tau = sqrt(2)) on the 4^4 lattice, with the
seeded synthetic inputs of paper_1805_03560_gb300.inputs.  kappa = 0.12 in
place of the paper's 0.1575: on this synthetic field the roots' series in K
converge only for a spectral radius of K below one.  Calls only oracle/ (and
the input generators); the GPU test compares the library's trajectory with
these numbers.  Run: python tests/golden/make_rooted_paper_set.py"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import coeffs as C  # noqa: E402
from paper_1805_03560_gb300 import inputs as I  # noqa: E402

L = (4, 4, 4, 4)
K, N, DEGS, N_T = 2, 8, (16, 42), 160
SAMPLE = [(s, mu) for s in (0, 17, 63, 128, 200, 255) for mu in (0, 3)]


def params():
    alpha, b, polys = C.rooted_coeffs(K, N, DEGS, N_T)
    return dict(beta=5.6, kappa=0.12, tau=math.sqrt(2.0), n_md=4, n_gauge=1, filter_k=K,
                n_t=N_T, n_max=N_T, b=b, alpha=alpha, c=C.heatbath_coeffs(K, N_T),
                root_polys=polys, root_N=N, level_steps=[40, 3, 2],
                term_level=[1] * N + [2] * N + [3], integrator=0)


def main():
    kw = params()
    U = I.gauge_links(L, 0.3, 1)
    P = I.momenta(L, 3)
    eta = np.stack([I.gaussian_half(L, 40 + j) for j in range(2 * N + 1)])
    _, r, Uo, _ = oracle.trajectory(L, U, P, eta, 0.5, tol_md=1e-13, tol_action=1e-14, **kw)
    out = {"citation": "Sec. IV.B, the rooted kappa^4 run (N = 8, n_1 = 16, n_2 = 42, n_t = 160, "
                       "m = 4, m_2 = 2, m_1 = 3, m_0 = 40, tau = sqrt(2)); kappa 0.12 on the "
                       "synthetic 4^4 field",
           "lattice": L, "links": "inputs.gauge_links(L, 0.3, 1)", "momenta": "inputs.momenta(L, 3)",
           "sources": "inputs.gaussian_half(L, 40 + j), j < 17", "tol_md": 1e-13,
           "tol_action": 1e-14,
           "params": {k: v for k, v in kw.items()},
           "H0": r["H0"], "H1": r["H1"], "dH": r["dH"], "plaq1": r["plaq1"],
           "U_end_sample": [[s, mu, [[z.real, z.imag] for z in Uo[s, mu].reshape(-1)]]
                            for s, mu in SAMPLE]}
    with open(os.path.join(HERE, "rooted_paper_set.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
