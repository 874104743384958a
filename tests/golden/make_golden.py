"""Writes oracle_regression.json: outputs of the FP64 oracle (oracle/ only, plus the
seeded input generators) on small fixed inputs. The paper prints no worked numerical
example, so these values pin the oracle against unintended change, not against the
paper; the pins in tests/test_oracle_*.py tie it to the paper's definitions.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ptc, staggered, wilson  # noqa: E402
from oracle import solvers as osolv  # noqa: E402
from paper_1109_2935_gb300 import synth  # noqa: E402

SITES = [[0, 0, 0, 0], [1, 0, 1, 1], [0, 1, 1, 3], [1, 1, 1, 2]]


def cvals(a):
    a = np.asarray(a).reshape(-1)
    return [[float(v.real), float(v.imag)] for v in a]


def at_sites(f, sites):
    return [cvals(f[t, z, y, x]) for x, y, z, t in sites]


def main():
    out = {}
    # Eq. 2, kappa form with the clover term, 2^3x4
    dims = (2, 2, 2, 4)
    U = synth.wilson_gauge(dims, 0.5, 1, 7001).numpy()
    A = wilson.clover(U, 1.0)
    psi = synth.wilson_spinor(dims, 7002).numpy()
    M = wilson.apply_M(U, A, 0.12, psi)
    out["wilson_clover_M"] = {
        "cite": "Eq. 2 (kappa form, clover from plaquette leaves), dims 2x2x2x4, kappa 0.12, c_sw 1, "
                "gauge seed 7001 (sigma 0.5, 1 smoothing step), spinor seed 7002",
        "norm2": float(np.vdot(M, M).real), "dot_psi_M": cvals(np.vdot(psi, M)),
        "sites_xyzt": SITES, "values": at_sites(M, SITES)}
    Md = wilson.apply_M(U, A, 0.12, psi, dagger=True)
    out["wilson_clover_Mdagger"] = {"cite": "M^dagger of the same", "norm2": float(np.vdot(Md, Md).real),
                                    "values": at_sites(Md, SITES)}
    S = wilson.apply_schur(U, A, 0.12, psi)
    out["wilson_schur_even"] = {"cite": "Sec. 3.1 even-odd Schur complement of the same",
                                "norm2": float(np.vdot(S, S).real)}
    # Eq. 3 asqtad, 4^4
    dims4 = (4, 4, 4, 4)
    fat, lng = (t.numpy() for t in synth.asqtad_links(dims4, 7003, 7004))
    chi = synth.staggered_spinor(dims4, 7005).numpy()
    N = staggered.apply_normal(fat, lng, 0.05, chi)
    out["asqtad_normal"] = {"cite": "Eq. 3, M^dagger M with m = 0.05, dims 4^4, fat/long seeds 7003/7004, "
                                    "source seed 7005",
                            "norm2": float(np.vdot(N, N).real), "values": at_sites(N, SITES)}
    # Sec. 3.2 / 8.1 Schwarz block MR, 4^4 lattice, 2^4 blocks, 4 steps
    U4 = synth.wilson_gauge(dims4, 0.5, 1, 7006).numpy()
    A4 = wilson.clover(U4, 1.0)
    b4 = synth.wilson_spinor(dims4, 7007).numpy()
    K = osolv.schwarz_mr(U4, A4, 0.12, b4, (2, 2, 2, 2), 4)
    out["schwarz_mr"] = {"cite": "Sec. 3.2 / Sec. 8.1 additive Schwarz, 2^4 blocks, 4 MR steps, kappa 0.12, "
                                 "gauge seed 7006, source seed 7007",
                         "norm2": float(np.vdot(K, K).real), "values": at_sites(K, SITES)}
    # learned preconditioner (extension): one forward pass of a 1-2-1 network
    W = [w.numpy() for w in synth.ptc_weights((1, 2, 1), 7008)]
    k, _ = ptc.net_forward(U4, W, b4)
    out["ptc_forward"] = {"cite": "parallel-transport convolution network 1-2-1 (extension), weights seed 7008, "
                                  "links and input as schwarz_mr",
                          "norm2": float(np.vdot(k, k).real), "values": at_sites(k, SITES)}
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
