"""The oracle reproduces its stored regression fixtures (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py from the oracle alone). A change in the oracle's
arithmetic shows up here first; it must then be justified by the paper's passage (or a
stated reading of it) and the fixtures rewritten by the script. CPU only."""
import json
import os

import numpy as np

from oracle import ptc, staggered, wilson
from oracle import solvers as osolv
from paper_1109_2935_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


def _check(name, field, sites=None):
    g = G[name]
    n2 = float(np.vdot(field, field).real)
    assert abs(n2 - g["norm2"]) <= 1e-12 * g["norm2"], name
    if "values" in g:
        sites = g.get("sites_xyzt", G["wilson_clover_M"]["sites_xyzt"])
        scale = np.sqrt(g["norm2"] / np.prod(field.shape[:4]))  # rms magnitude per site
        for (x, y, z, t), vals in zip(sites, g["values"]):
            got = field[t, z, y, x].reshape(-1)
            ref = np.array([complex(a, b) for a, b in vals])
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale, name


def test_wilson_fixtures():
    dims = (2, 2, 2, 4)
    U = synth.wilson_gauge(dims, 0.5, 1, 7001).numpy()
    A = wilson.clover(U, 1.0)
    psi = synth.wilson_spinor(dims, 7002).numpy()
    M = wilson.apply_M(U, A, 0.12, psi)
    _check("wilson_clover_M", M)
    d = np.vdot(psi, M)
    ref = complex(*G["wilson_clover_M"]["dot_psi_M"][0])
    assert abs(d - ref) <= 1e-12 * abs(ref)
    _check("wilson_clover_Mdagger", wilson.apply_M(U, A, 0.12, psi, dagger=True))
    _check("wilson_schur_even", wilson.apply_schur(U, A, 0.12, psi))


def test_asqtad_schwarz_ptc_fixtures():
    dims4 = (4, 4, 4, 4)
    fat, lng = (t.numpy() for t in synth.asqtad_links(dims4, 7003, 7004))
    chi = synth.staggered_spinor(dims4, 7005).numpy()
    _check("asqtad_normal", staggered.apply_normal(fat, lng, 0.05, chi))
    U4 = synth.wilson_gauge(dims4, 0.5, 1, 7006).numpy()
    A4 = wilson.clover(U4, 1.0)
    b4 = synth.wilson_spinor(dims4, 7007).numpy()
    _check("schwarz_mr", osolv.schwarz_mr(U4, A4, 0.12, b4, (2, 2, 2, 2), 4))
    W = [w.numpy() for w in synth.ptc_weights((1, 2, 1), 7008)]
    k, _ = ptc.net_forward(U4, W, b4)
    _check("ptc_forward", k)
