"""Eccentric-charge sphere study of Sec. 3.3 (Fig. 4c-f), regenerated on icospheres: radius 1 A,
one +1 e charge moved from the centre toward the surface, kappa = 1, eps = 80, HOBI-PB and
LOBI-PB against the Kirkwood series, surface-potential error e_phi (Eq. (24)) per
icosahedral level. The figure's data are not in the paper; the test checks the paper's
observations that hold on uniform meshes, and writes the table as JSON into the directory named
by the environment variable HOBI_STUDY_OUT when it is set."""
import json
import os

import numpy as np
import pytest

from oracle import kirkwood as kw
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu

R, KAPPA, EPS1, EPS2 = 1.0, 1.0, 1.0, 80.0
POSITIONS = (0.0, 0.3, 0.5, 0.7, 0.9)
LEVELS = (1, 2, 3, 4, 5)


def _ephi(V, F, N, Q, scheme):
    s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision="fp64", scheme=scheme)
    phi, _, info = s.solve(1e-10, 300)
    if scheme == "lobi":
        pts, _, _ = s.nodes()
        pts = pts / np.linalg.norm(pts, axis=1, keepdims=True) * R  # centroid -> nearest sphere point
    else:
        pts = V
    exact, _ = kw.surface_potential(pts, Q, R, EPS1, EPS2, KAPPA)
    s.close()
    return float(np.max(np.abs(phi - exact)) / np.max(np.abs(exact))), info["iterations"]


@pytest.fixture(scope="module")
def table():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = {}
    for L in LEVELS:
        V, F, N = synth.icosphere(L, R)
        for x in POSITIONS:
            Q = synth.point_charge(x, 0.0, 0.0, 1.0)
            for scheme in ("hobi", "lobi"):
                out[(scheme, L, x)] = _ephi(V, F, N, Q, scheme)
    out_dir = os.environ.get("HOBI_STUDY_OUT")
    if out_dir and os.path.isdir(out_dir):
        rows = [{"scheme": k[0], "level": k[1], "faces": 20 * 4 ** k[1], "x": k[2], "e_phi": v[0],
                 "iterations": v[1]} for k, v in sorted(out.items())]
        with open(os.path.join(out_dir, "eccentric_sphere_study.json"), "w") as fh:
            json.dump(rows, fh, indent=1)
    return out


def test_hobi_more_accurate_for_interior_charges(table):
    """Observation (1) of Sec. 3.3: HOBI errors are smaller than LOBI's."""
    for L in LEVELS[1:]:
        for x in (0.0, 0.3, 0.5):
            assert table[("hobi", L, x)][0] < table[("lobi", L, x)][0], (L, x)


def _slope(table, scheme, x, levels=(2, 3, 4, 5)):
    """Least-squares order in the density d (x4 per level); HOBI's pattern is irregular near the
    surface (Sec. 3.3, observation (2)), so two-level ratios can mislead."""
    e = np.log([table[(scheme, L, x)][0] for L in levels])
    return -np.polyfit(np.log(4.0) * np.array(levels), e, 1)[0]


def test_hobi_converges_faster(table):
    """Fig. 4e/f: a steeper error-vs-elements slope for HOBI than for LOBI; LOBI near half order."""
    for x in (0.0, 0.5, 0.9):
        sh, sl = _slope(table, "hobi", x), _slope(table, "lobi", x)
        assert sh > sl > 0.2, (x, sh, sl)
    assert 0.3 < _slope(table, "lobi", 0.5) < 0.9


def test_errors_fall_with_refinement_and_grow_near_surface(table):
    for scheme in ("hobi", "lobi"):
        for x in POSITIONS:
            assert table[(scheme, 5, x)][0] < table[(scheme, 2, x)][0]
        # a charge close to the interface is harder (Sec. 3.3): at every level
        for L in LEVELS:
            assert table[(scheme, L, 0.9)][0] > table[(scheme, L, 0.0)][0]
