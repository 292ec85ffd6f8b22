"""CPU checks of the C ABI: the library loads, exports every symbol its headers
declare, and rejects invalid arguments and geometries before touching the GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2406_15959_gb300 import elm_ddm as E
from paper_2406_15959_gb300 import workload as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(elm_(?:ddm|mlp)_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = E.load()
    names = declared_symbols()
    assert {"elm_ddm_setup", "elm_ddm_assemble", "elm_ddm_schur", "elm_ddm_solve"} <= names
    for name in names:
        assert hasattr(lib, name), name
    from paper_2406_15959_gb300 import mlp as M
    assert set(E.SYMBOLS) | set(M.SYMBOLS) >= names


def _setup(desc, counts, xy, nrm, dof):
    lib = E.load()
    h = ctypes.c_void_p()
    rc = lib.elm_ddm_setup(ctypes.byref(desc), counts.ctypes.data, xy.ctypes.data,
                           nrm.ctypes.data, dof.ctypes.data, None, ctypes.byref(h))
    return rc, lib.elm_ddm_last_error(None).decode(), h


def _arrays(g):
    ga = E.GeometryArrays.from_geometry(g)
    return ga.counts.copy(), ga.xy.copy(), ga.nrm.copy(), ga.dof.copy()


def _desc(g, n, **kw):
    d = dict(n_sub=g.n_sub, n_neurons=n, m_max=g.m_max, n_gamma=g.n_gamma, op=0, max_rhs=1)
    d.update(kw)
    return E.Desc(**d)


G = wl.make_geometry(3, 2, 4, 4, 3, 3)


@pytest.mark.parametrize("kw,msg", [
    (dict(n_sub=0), "must be >= 1"),
    (dict(op=7), "unsupported operator"),
    (dict(max_rhs=65), "max_rhs"),
    (dict(n_neurons=10_000), "8192"),
    (dict(n_neurons=40), "fewer rows than neurons"),
    (dict(n_gamma=G.n_gamma + 1), "not shared by exactly two"),
    (dict(flags=128), "unknown flags"),
    (dict(flags=E.FLAG_BLOCK_JACOBI | E.FLAG_SCHUR_CG), "assembled S"),
    (dict(flags=E.FLAG_BLOCK_JACOBI | E.FLAG_MIXED), "assembled S"),
    (dict(flags=E.FLAG_MIXED | E.FLAG_FP64_SIMT), "tensor-core back end"),
    (dict(flags=E.FLAG_MIXED | E.FLAG_SCHUR_CG), "direct Schur solve"),
])
def test_setup_rejects_bad_descriptors(kw, msg):
    c, xy, nrm, dof = _arrays(G)
    rc, err, h = _setup(_desc(G, 8, **kw), c, xy, nrm, dof)
    assert rc == E.ERR_ARG and msg in err and not h.value


def test_setup_rejects_unshared_interface_unknown():
    c, xy, nrm, dof = _arrays(G)
    s = 0
    r0 = c[s, 0] + c[s, 1]
    dof[s, r0] = (dof[s, r0] + 1) % G.n_gamma          # now one unknown has 3 owners, one has 1
    rc, err, _ = _setup(_desc(G, 8), c, xy, nrm, dof)
    assert rc == E.ERR_ARG and "exactly two" in err


def test_setup_rejects_mismatched_edges():
    c, xy, nrm, dof = _arrays(G)
    # reverse the order of one edge's unknowns in one subdomain only
    s = 1
    r0 = c[s, 0] + c[s, 1]
    dof[s, r0:r0 + 3] = dof[s, r0:r0 + 3][::-1].copy()
    rc, err, _ = _setup(_desc(G, 8), c, xy, nrm, dof)
    assert rc == E.ERR_ARG and "edges" in err


def test_setup_rejects_nonfinite_points():
    c, xy, nrm, dof = _arrays(G)
    xy[2, 1, 0] = np.nan
    rc, err, _ = _setup(_desc(G, 8), c, xy, nrm, dof)
    assert rc == E.ERR_NONFINITE


def test_setup_rejects_interface_rows_on_single_domain():
    g = wl.make_geometry(1, 1, 4, 4, 3, 3)
    c, xy, nrm, dof = _arrays(g)
    c[0, 2] = 1
    rc, err, _ = _setup(_desc(g, 8), c, xy, nrm, dof)
    assert rc == E.ERR_ARG


def test_null_handle_calls_fail_cleanly():
    lib = E.load()
    assert lib.elm_ddm_schur(None) == E.ERR_ARG
    assert lib.elm_ddm_assemble(None, None, None) == E.ERR_ARG
    assert lib.elm_ddm_solve(None, None, 1, None, None) == E.ERR_ARG
    assert lib.elm_ddm_check(None) == E.ERR_ARG
    assert lib.elm_ddm_destroy(None) == E.ERR_ARG


def test_new_entry_points_reject_null_handles():
    lib = E.load()
    assert lib.elm_ddm_get_points(None, 0, None, None) == E.ERR_ARG
    assert lib.elm_ddm_set_wait_limit(None, 1.0, 0) == E.ERR_ARG


def test_setup_checks_per_subdomain_neuron_counts():
    c, xy, nrm, dof = _arrays(G)
    lib = E.load()
    for ns, msg in [(0, "not in 1..n_neurons"), (9, "not in 1..n_neurons")]:
        c4 = np.ascontiguousarray(np.concatenate([c, np.full((G.n_sub, 1), ns, np.int32)], 1))
        h = ctypes.c_void_p()
        d = _desc(G, 8, flags=E.FLAG_NEURONS_PER_SUB)
        rc = lib.elm_ddm_setup(ctypes.byref(d), c4.ctypes.data, xy.ctypes.data, nrm.ctypes.data,
                               dof.ctypes.data, None, ctypes.byref(h))
        assert rc == E.ERR_ARG and msg in lib.elm_ddm_last_error(None).decode()


# ---- explicit A-rows (elm_ddm_setup_flux; the corner rule at cross points) ----

GX = wl.make_paper_grid_geometry(3, 13, cross_points=True)


def _setup_flux(desc, g, flux):
    lib = E.load()
    ga = E.GeometryArrays.from_geometry(g)
    f = flux
    fd = E.FluxRowsDesc(int(f.n_flux), int(f.row.shape[1]), f.count.ctypes.data, f.row.ctypes.data,
                        f.nrm.ctypes.data, f.fdof.ctypes.data)
    h = ctypes.c_void_p()
    rc = lib.elm_ddm_setup_flux(ctypes.byref(desc), ga.counts.ctypes.data, ga.xy.ctypes.data,
                                ga.nrm.ctypes.data, ga.dof.ctypes.data, ctypes.byref(fd), None, ctypes.byref(h))
    return rc, lib.elm_ddm_last_error(None).decode(), h


def _flux_copy(g):
    f = g.flux
    return type(f)(f.n_flux, f.count.copy(), f.row.copy(), f.nrm.copy(), f.fdof.copy())


def test_cross_points_need_explicit_flux_rows():
    """Unknowns shared by four subdomains: elm_ddm_setup (one A-row per interface row)
    rejects them before any CUDA call."""
    c, xy, nrm, dof = _arrays(GX)
    rc, err, h = _setup(_desc(GX, 8), c, xy, nrm, dof)
    assert rc == E.ERR_ARG and "exactly two" in err and not h.value


@pytest.mark.parametrize("flags", [E.FLAG_SCHUR_CG, E.FLAG_MIXED, E.FLAG_BLOCK_JACOBI])
def test_setup_flux_rejects_the_cg_and_mixed_modes(flags):
    rc, err, h = _setup_flux(_desc(GX, 8, flags=flags), GX, _flux_copy(GX))
    assert rc == E.ERR_ARG and "explicit flux rows" in err and not h.value


def test_setup_flux_rejects_bad_rows():
    f = _flux_copy(GX)
    f.row[4, 0] = GX.counts[4, 2]                      # past the interface rows
    rc, err, _ = _setup_flux(_desc(GX, 8), GX, f)
    assert rc == E.ERR_ARG and "out of range" in err
    f = _flux_copy(GX)
    f.fdof[4, 0] = f.fdof[4, 1]                        # one condition with three rows, one with one
    rc, err, _ = _setup_flux(_desc(GX, 8), GX, f)
    assert rc == E.ERR_ARG and "exactly two" in err
    f = _flux_copy(GX)
    k = int(f.count[0])
    f.fdof[0, :k] = f.fdof[0, :k][::-1].copy()           # same conditions, mismatched order
    f.row[0, :k] = f.row[0, :k][::-1].copy()
    rc, err, _ = _setup_flux(_desc(GX, 8), GX, f)
    assert rc == E.ERR_ARG and "matching groups" in err
    f = _flux_copy(GX)
    f.nrm[2, 3, 1] = np.inf
    rc, err, _ = _setup_flux(_desc(GX, 8), GX, f)
    assert rc == E.ERR_NONFINITE
