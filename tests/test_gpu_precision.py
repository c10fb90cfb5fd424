"""Precision study: float32 projections with a compensated (Kahan / TwoSum)
float32 z, the same without compensation, and the deterministic fixed-point
back-projection, each against the FP64 oracle after the same epochs.  Reports
the image relative L2 error, the z error and the objective gap; all must be
inside the image tolerance."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2201_05497_gb300 import synth as S
from tests import _helpers as H
from tests.test_gpu_lmspdhg import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    from paper_2201_05497_gb300 import build, lm as _lm
    build.build()
    _lm.load_library()
    return _lm


def test_precision_modes_against_fp64(lm):
    c = Case(lm, "3d_mid")
    epochs = 3
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * epochs, seed=3)
    o = c.oracle()
    o.run(seq)
    f_o = o.objective()
    res = {}
    for name, kw in [("fp32+kahan", dict(kahan=True)), ("fp32", dict(kahan=False)),
                     ("fp32+kahan deterministic", dict(kahan=True, deterministic=True))]:
        g = c.gpu(**kw)
        for k in range(epochs):
            g.epoch(seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)])
        x, z = g.x().cpu().numpy(), g.z().cpu().numpy()
        f = g.objective()
        res[name] = {"x_rel_l2": H.rel_l2(x, o.x), "z_rel_l2": H.rel_l2(z, o.z),
                     "objective_rel_gap": (f - f_o) / abs(f_o)}
        g.close()
    print("PRECISION_STUDY " + json.dumps(res))
    for name, r in res.items():
        assert r["x_rel_l2"] < H.REL_L2_IMAGE, (name, r)
        assert r["z_rel_l2"] < H.REL_L2_IMAGE, (name, r)
        assert abs(r["objective_rel_gap"]) < 1e-5, (name, r)


def test_2d_config_20_epochs(lm):
    """The 2D configuration as stated: 256 crystals, 128^2 image, 2e5 events,
    28 subsets, 20 epochs, TV beta = 0.03."""
    c = Case(lm, "2d")
    o = c.oracle()
    g = c.gpu()
    E = 20
    seq = S.selection_sequence(c.n_sub, 2 * c.n_sub * E, seed=3)
    for k in range(E):
        s = seq[2 * c.n_sub * k:2 * c.n_sub * (k + 1)]
        g.epoch(s)
        o.run(s)
    err = H.rel_l2(g.x().cpu().numpy(), o.x)
    print(f"2D_20_EPOCHS x_rel_l2={err:.3e}")
    assert err < H.REL_L2_IMAGE
