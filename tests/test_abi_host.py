"""Host-side checks of the C ABI (no GPU): library loads, every declared entry
point is exported, the library's tableau builder agrees with the oracle's, and
malformed input is rejected before any device work."""
import os
import re

import numpy as np
import pytest

import paper_2507_04991_gb300 as pk
import workloads
from oracle import tableau as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return pk.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "perrk.h")).read()
    declared = set(re.findall(r"\b(perrk_[a-z_0-9]+)\s*\(", hdr))
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(pk.EXPORTED) == declared


@pytest.mark.parametrize("p,E", [(2, [8, 4]), (2, [16, 12, 8, 4, 2]), (3, [12, 6, 3]), (3, [8, 4]), (3, [3]),
                                 (4, [16, 10, 7, 5]), (4, [5]), (2, [2])])
def test_tableau_builder_matches_oracle(lib, p, E):
    c, b, a1, asub = pk.perrk_build_tableau(p, E)
    oc, ob, As = T.family(p, E)
    S = len(oc)
    assert np.abs(c - oc).max() < 1e-15 and np.abs(b - ob).max() == 0.0
    for r, A in enumerate(As):
        for i in range(1, S):
            full = np.zeros(S)
            full[0] += a1[r, i]
            full[i - 1] += asub[r, i]
            assert np.abs(full - A[i]).max() < 1e-15, (r, i)


def _small_mesh():
    wl = workloads.small_box_2d(n=4, seed=1, R=2, E=[6, 3], order=3)
    keep = pk._Keep()
    m = pk.mesh_desc(wl.coords, wl.faces, wl.part, keep)
    tab = pk.perrk_build_tableau(3, [6, 3])
    return wl, keep, m, tab


@pytest.mark.parametrize("breakage", ["bad_rowsum", "bad_E", "bad_part", "bad_face", "missing_face", "bad_b", "bad_N",
                                      "asub_inactive"])
def test_invalid_input_rejected(lib, breakage):
    wl, keep, m, (c, b, a1, asub) = _small_mesh()
    c, b, a1, asub = c.copy(), b.copy(), a1.copy(), asub.copy()
    E = [6, 3]
    part = wl.part.copy()
    faces = wl.faces.copy()
    if breakage == "bad_rowsum":
        a1[0, 3] += 1e-6
    elif breakage == "bad_E":
        E = [6, 2]
    elif breakage == "bad_part":
        part[0] = 5
    elif breakage == "bad_face":
        faces[0, 3] = 2
    elif breakage == "missing_face":
        faces = faces[1:]          # one element face pair left without partner
    elif breakage == "bad_b":
        b[1] = 0.1
    elif breakage == "asub_inactive":
        asub[1, 2] = 0.01
        a1[1, 2] -= 0.01
    m = pk.mesh_desc(wl.coords, faces, part, keep)
    if breakage == "bad_N":
        m.N = 4
    s = pk.scheme_desc(3, E, c, b, a1, asub, pk.EULER_2D, pk.SURFACE_ES_RUSANOV, 1.4, keep)
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_create(m, s, pk.options())
    assert ei.value.status == pk.PERRK_INVALID_ARG
    assert pk.last_error()


def test_tableau_below_archetype_minimum_rejected(lib):
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_build_tableau(3, [6, 4, 2])
    assert ei.value.status == pk.PERRK_INVALID_ARG
    assert "archetype minimum" in pk.last_error()


def test_status_strings(lib):
    assert pk.status_string(0) == "ok"
    assert pk.status_string(3) == "non-physical state"
    assert pk.perrk_mlp_size() == 64 * 6 + 64 + 64 * 64 + 64 + 64 + 1 + 2 * 6 + 1


@pytest.mark.parametrize("bad", ["solver", "bracket"])
def test_invalid_solver_options_rejected(lib, bad):
    wl, keep, m, (c, b, a1, asub) = _small_mesh()
    s = pk.scheme_desc(3, [6, 3], c, b, a1, asub, pk.EULER_2D, pk.SURFACE_ES_RUSANOV, 1.4, keep)
    o = pk.options(solver=pk.SOLVER_BISECTION, bracket=(1.2, 0.8)) if bad == "bracket" else pk.options()
    if bad == "solver":
        o.solver = 7
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_create(m, s, o)
    assert ei.value.status == pk.PERRK_INVALID_ARG


@pytest.mark.parametrize("case", sorted(pk.NEWTON_PRESETS))
def test_newton_presets_accepted(lib, case):
    """The paper's per-case root-finder settings are valid options (create accepts them)."""
    wl, keep, m, (c, b, a1, asub) = _small_mesh()
    s = pk.scheme_desc(3, [6, 3], c, b, a1, asub, pk.EULER_2D, pk.SURFACE_ES_RUSANOV, 1.4, keep)
    o = pk.options_preset(case)
    assert o.newton_max_it == pk.NEWTON_PRESETS[case]["max_it"]
    try:
        h = pk.perrk_create(m, s, o)
    except pk.PerrkError as err:
        # on a machine without a GPU, create stops at the first device allocation
        assert err.status == pk.PERRK_CUDA_ERROR or err.status == pk.PERRK_OUT_OF_MEMORY
        return
    pk.perrk_destroy(h)


def test_header_compiles_as_c(tmp_path):
    """include/perrk.h is a C header: it compiles as strict C11 and its
    checkpoint records have the sizes the binding assumes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "perrk.h"\n'
                   'int main(void) {\n'
                   '  _Static_assert(sizeof(perrk_checkpoint_header) == 40, "header");\n'
                   '  _Static_assert(sizeof(perrk_resume_info) == 96, "resume");\n'
                   '  return 0;\n}\n')
    out = tmp_path / "h.o"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert pk.C.sizeof(pk.perrk_checkpoint_header) == 40 and pk.C.sizeof(pk.perrk_resume_info) == 96


def _mortar_mesh():
    wl = workloads.quadtree_patch_2d(n=8, depth=1, E=(6, 3), order=3)
    keep = pk._Keep()
    tab = pk.perrk_build_tableau(3, [6, 3])
    return wl, keep, tab


@pytest.mark.parametrize("breakage", ["swapped_halves", "face_twice", "missing_mortar", "index_range"])
def test_invalid_mortars_rejected(lib, breakage):
    """Malformed 2:1 mortar rows are refused before any device work."""
    wl, keep, (c, b, a1, asub) = _mortar_mesh()
    mortars = wl.mortars.copy()
    faces = wl.faces
    if breakage == "swapped_halves":
        mortars[0, [2, 3]] = mortars[0, [3, 2]]
    elif breakage == "face_twice":
        mortars = np.concatenate([mortars, mortars[:1]])
    elif breakage == "missing_mortar":
        mortars = mortars[1:]
    else:
        mortars[0, 2] = wl.n_elem
    m = pk.mesh_desc(wl.coords, faces, wl.part, keep, mortars)
    s = pk.scheme_desc(3, [6, 3], c, b, a1, asub, pk.EULER_2D, pk.SURFACE_ES_RUSANOV, 1.4, keep)
    with pytest.raises(pk.PerrkError) as ei:
        pk.perrk_create(m, s, pk.options())
    assert ei.value.status == pk.PERRK_INVALID_ARG, pk.last_error()
    assert pk.last_error()


def test_valid_mortar_mesh_passes_validation(lib):
    """A well-formed quadtree mesh passes the host checks (without a GPU the
    call then stops at the first device allocation)."""
    wl, keep, (c, b, a1, asub) = _mortar_mesh()
    m = pk.mesh_desc(wl.coords, wl.faces, wl.part, keep, wl.mortars)
    s = pk.scheme_desc(3, [6, 3], c, b, a1, asub, pk.EULER_2D, pk.SURFACE_ES_RUSANOV, 1.4, keep)
    try:
        h = pk.perrk_create(m, s, pk.options())
    except pk.PerrkError as err:
        assert err.status in (pk.PERRK_CUDA_ERROR, pk.PERRK_OUT_OF_MEMORY), pk.last_error()
        return
    pk.perrk_destroy(h)
