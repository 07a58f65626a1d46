"""Host-side checks of the CUDA library (no GPU): the C ABI loads and exports
every declared symbol, and the subdomain systems it packs for the GPU
(SELL-32 arrays, Robin entries, loads, face masses) unpack to the oracle's
matrices entry by entry."""
import re
from pathlib import Path

import numpy as np
import pytest

import gen
import oracle

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def osm():
    from paper_2112_03851_gb300 import build
    build.build()
    import paper_2112_03851_gb300 as pkg
    pkg.load()
    return pkg


def test_header_symbols_are_exported(osm):
    header = (ROOT / "include" / "osm.h").read_text()
    declared = set(re.findall(r"^(?:osm_status|void|const char \*)\s*(osm_\w+)\(", header, re.M))
    declared |= set(re.findall(r"\n(?:osm_status|void|const char \*)\s*(osm_\w+)\(", header))
    assert len(declared) >= 20
    lib = osm.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert set(osm.EXPORTED) == declared


def test_status_strings(osm):
    lib = osm.load()
    assert lib.osm_status_string(0) == b"ok"
    assert lib.osm_status_string(4) == b"iteration cap reached"


def test_log_uniform_p_matches_independent_splitmix(osm):
    for seed, lo, hi in [(0, 0.5, 200.0), (7, 2.0, 50.0)]:
        a = osm.log_uniform_p(seed, 64, lo, hi)
        b = gen.log_uniform_p(seed, 64, lo, hi)
        assert np.all(a >= lo) and np.all(a <= hi)
        assert np.allclose(a, b, rtol=4e-16, atol=0)


CASES = {
    "sphere8_2x2x2": lambda: gen.sphere_problem(8, 2, 10.0),
    "regional_uneven": lambda: gen.regional_problem(nx=12, ny=10, nz=8, sx=3, sy=2, sz=2, p=2.0,
                                                    seed=4, lx=10.0, ly=8.0, lz=3.0),
    "layered_3x1x2": lambda: gen.layered_problem(n=6, s=1, seed=2, n_spheres=4),
}


def _with_cuts(prob, name):
    if name == "layered_3x1x2":
        prob.cx = np.array([0, 2, 3, 6], dtype=np.int32)
        prob.cz = np.array([0, 4, 6], dtype=np.int32)
    return prob


@pytest.mark.parametrize("name", sorted(CASES))
def test_local_systems_match_oracle(osm, name):
    prob = _with_cuts(CASES[name](), name)
    p = 3.7
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, p)
    for s in range(S.nsub):
        A_ref, f_ref, g_ref, _ = S.sub_export(s)
        A, f = osm.host_local_system(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, p, s)
        assert A.shape == A_ref.shape
        D = (A - A_ref).toarray()
        assert np.abs(D).max() <= 1e-13 * np.abs(A_ref).max(), (s, np.abs(D).max())
        assert np.abs(f - f_ref).max() <= 1e-13 * max(np.abs(f_ref).max(), 1e-300), s


@pytest.mark.parametrize("name", sorted(CASES))
def test_face_masses_match_oracle(osm, name):
    prob = _with_cuts(CASES[name](), name)
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, 1.0)
    for f in range(S.nface):
        g_ref, M_ref = S.face_export(f)
        g, M = osm.host_face_system(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, f)
        assert np.array_equal(g, g_ref), f
        assert np.abs((M - M_ref).toarray()).max() <= 1e-15 * np.abs(M_ref).max(), f


@pytest.mark.parametrize("name", sorted(CASES))
def test_second_order_local_systems_and_face_stiffness_match_oracle(osm, name):
    """Split transmission entries (lower/upper side, face mass and tangential
    stiffness) reassembled with unsymmetric oo2 coefficients equal the
    oracle's local matrices; every face stiffness equals the oracle's."""
    prob = _with_cuts(CASES[name](), name)
    tc = (1.3, 0.21, 0.4, 0.77)
    S = oracle.Schwarz(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, tc=tc)
    for s in range(S.nsub):
        A_ref, _, _, _ = S.sub_export(s)
        A, _ = osm.host_local_system(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, 0.0, s, tc=tc)
        assert np.abs((A - A_ref).toarray()).max() <= 1e-13 * np.abs(A_ref).max(), s
    for f in range(S.nface):
        S_ref = S.face_stiffness_export(f)
        _, Sf = osm.host_face_stiffness(prob.xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, f)
        assert np.abs((Sf - S_ref).toarray()).max() <= 1e-14 * np.abs(S_ref).max(), f


def test_bad_inputs_are_rejected(osm):
    prob = gen.sphere_problem(4, 2, 1.0)
    with pytest.raises(osm.OsmError):
        osm.host_local_system(prob.xc, prob.yc, prob.zc, prob.drho, [0, 3, 2, 4], prob.cy, prob.cz, 1.0, 0)
    xc = prob.xc.copy()
    xc[2] = xc[1]
    with pytest.raises(osm.OsmError):
        osm.host_local_system(xc, prob.yc, prob.zc, prob.drho, prob.cx, prob.cy, prob.cz, 1.0, 0)
    d = prob.drho.copy()
    d[3] = np.nan
    with pytest.raises(osm.OsmError):
        osm.host_local_system(prob.xc, prob.yc, prob.zc, d, prob.cx, prob.cy, prob.cz, 1.0, 0)
