"""Host tables of the symmetry-reduced FP64 M2L (paper_1712_07739_gb300/csrc/
cube_sym.h; Sec. 6: 16 of the 316 operators), checked without a GPU against
an independent construction.

tests/cube_sym_dump.cpp prints the library's tables; this test rebuilds what
each entry must be from the oracle's group (``oracle_b.cube_group``), its
orbits (``oracle_b.offset_orbits``) and numpy einsum:

* the 48 maps are the cube group, with their determinants;
* the 16 representatives are the oracle's orbit representatives, and every
  offset with max |o_i| >= 2 is its map applied to its representative (the
  others carry none);
* the component table applies det(g) rho(g) to a random 6 x 9 kernel exactly
  as the einsum form of K(g d) = det(g) g g g g K(d) does;
* the frequency table gives g^T f (mod N) for every frequency of N = 14;
* the invariance check accepts isotropic and aligned cubic media and refuses
  a turned crystal.
"""
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import oracle_b as ob
from paper_1712_07739_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("cube_sym") / "cube_sym_dump")
    subprocess.check_call([gxx, "-std=c++17", "-O1", "-Wall", "-o", out, os.path.join(HERE, "cube_sym_dump.cpp")])
    return out


@pytest.fixture(scope="module")
def tables(exe):
    txt = subprocess.run([exe, "tables"], check=True, capture_output=True, text=True).stdout
    maps, reps, offs, gmap = {}, {}, {}, {}
    for line in txt.splitlines():
        w = line.split()
        v = [int(x) for x in w[1:]]
        if w[0] == "map":
            maps[v[0]] = v[1:]
        elif w[0] == "rep":
            reps[v[0]] = v[1]
        elif w[0] == "off":
            offs[v[0]] = v[1]
        elif w[0] == "gmap":
            gmap[v[0]] = v[1:]
    return maps, reps, offs, gmap


def _g(entry):
    pi, s, det = entry[:3], entry[3:6], entry[6]
    g = np.zeros((3, 3), dtype=np.int64)
    for i in range(3):
        g[i, pi[i]] = s[i]
    return g, det


def _vec(oi):
    return (oi % 7 - 3, (oi // 7) % 7 - 3, oi // 49 - 3)


def test_maps_are_the_cube_group(tables):
    maps = tables[0]
    assert len(maps) == 48
    mine = {g.tobytes(): round(np.linalg.det(g)) for g in ob.cube_group()}
    seen = set()
    for gi, e in maps.items():
        g, det = _g(e)
        assert g.tobytes() in mine and mine[g.tobytes()] == det
        seen.add(g.tobytes())
    assert len(seen) == 48


def test_representatives_and_offsets(tables):
    maps, reps, offs, _ = tables
    want = {rep for rep, _ in ob.offset_orbits()}
    got = {_vec(reps[r]) for r in range(16)}
    assert got == want
    for oi in range(343):
        o = _vec(oi)
        code = offs[oi]
        if max(abs(x) for x in o) < 2:
            assert code == -1
            continue
        r, gi = code & 255, code >> 8
        g, _ = _g(maps[gi])
        assert tuple(g @ np.array(_vec(reps[r]))) == o


def _full(K):  # [6, 9] -> [3, 3, 3, 3]
    T = np.zeros((3, 3, 3, 3))
    for i, (a, b) in enumerate(VOIGT):
        T[a, b] = K[i].reshape(3, 3)
        T[b, a] = K[i].reshape(3, 3)
    return T


def test_component_table_is_det_rho(tables):
    maps, _, _, gmap = tables
    rng = np.random.default_rng(4)
    K = rng.normal(size=(6, 9))
    for gi in range(48):
        g, det = _g(maps[gi])
        want = det * np.einsum("ai,bj,wk,rl,ijkl->abwr", g, g, g, g, _full(K))
        tab = gmap[gi]
        for ab, (a, b) in enumerate(VOIGT):
            for wr in range(9):
                code = tab[ab * 9 + wr]
                src, neg = code & 63, bool(code & 64)
                got = -K.reshape(-1)[src] if neg else K.reshape(-1)[src]
                assert got == pytest.approx(want[a, b, wr // 3, wr % 3], abs=1e-14)


def test_frequency_table_is_gT_f(tables):
    maps, _, _, gmap = tables
    N = 14
    f = np.array(list(itertools.product(range(N), repeat=3)))
    for gi in range(48):
        g, _ = _g(maps[gi])
        want = (f @ g) % N  # (g^T f)_j = sum_i g_ij f_i
        tab = gmap[gi][54:57]
        got = np.zeros_like(f)
        for j in range(3):
            a = tab[j]
            v = f[:, a & 3]
            got[:, j] = np.where(a & 4, (N - v) % N, v)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("name,ok", [("iso", 1), ("cubic", 1), ("turned", 0)])
def test_invariance_check(exe, name, ok):
    import oracle

    C6 = {"iso": synth.isotropic_voigt(1.0, 0.3), "cubic": synth.cubic_voigt(),
          "turned": synth.rotated_voigt(synth.cubic_voigt(), synth.rotation())}[name]
    C = oracle.voigt_to_cijkl(C6).reshape(-1)
    out = subprocess.run([exe, "invariant"], input=" ".join(repr(float(c)) for c in C), check=True,
                         capture_output=True, text=True).stdout
    assert int(out) == ok
