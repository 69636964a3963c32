"""The default parameters of the library and of the oracle are the settings the
paper prints for its tests (tests/golden/paper_settings.json, each value with
its passage). No compute call: runs without a GPU."""
import json
import os

import numpy as np

import oracle as O
import paper_2304_09485_gb300 as H

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_settings.json")


def settings():
    with open(GOLDEN) as f:
        d = json.load(f)
    return {k: v["value"] for k, v in d.items() if not k.startswith("_")}


SCALARS = ("gamma", "tau_eps", "tau_C", "krylov_dim", "restarts", "jacobi_sweeps", "cfl", "lin_weight")


def test_every_setting_has_a_citation():
    with open(GOLDEN) as f:
        d = json.load(f)
    for k, v in d.items():
        if not k.startswith("_"):
            assert set(v) == {"value", "cite"} and v["cite"].startswith("Sec."), k


def test_library_defaults_are_the_papers_settings():
    s, p = settings(), H.hgks_default_params()
    for k in SCALARS:
        assert getattr(p, k) == s[k], k


def test_oracle_defaults_are_the_papers_settings():
    s, p = settings(), O.make_params()
    for k in SCALARS:
        assert getattr(p, k) == s[k], k


def test_central_weight_from_the_linear_weights():
    """gamma_0 = 1 - gamma_i M leaves the central polynomial the largest weight
    (0.9 for the four sub-stencils of a tetrahedron) and the weights summing to one."""
    s = settings()
    g = np.array([1 - s["lin_weight"] * s["sub_stencils_tet"]] + [s["lin_weight"]] * s["sub_stencils_tet"])
    assert abs(g.sum() - 1.0) < 1e-15 and g[0] == max(g)


def test_oracle_face_rule_has_the_printed_point_count():
    """The oracle evaluates the face flux at as many Gauss points per face as the setting."""
    from paper_2304_09485_gb300 import inputs as I
    om = O.OracleMesh(I.cavity_mesh(2))
    assert om.face_gauss_points(0, 0).shape == (settings()["gauss_points_per_face"], 3)
