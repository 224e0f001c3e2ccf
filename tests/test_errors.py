"""Error paths of the C ABI: every status code of include/mlev.h except MLEV_ETIMEOUT is
produced here and comes back with its message, and a context stays usable after a failed call.

Failures are made on the host: bad inputs, iteration caps of 1, a workspace that is too small,
and the library's MLEV_FAULT hooks (a planner allocation that fails, a table copy that fails,
a NaN planted in the staged coefficient after validation). None of them faults, traps or
hangs a GPU. MLEV_ETIMEOUT comes only from the bounded wait on a TMA transaction barrier,
which no test forces to expire (a bulk copy could still be in flight).
"""
import numpy as np
import pytest

import workloads as W
from paper_1401_4969_gb300 import mlev

EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, EUNSUPPORTED, ESTATE = -1, -2, -3, -4, -5, -6, -7


def _code(excinfo):
    return excinfo.value.code


# ------------------------------------------------------------------ host only (planning context)
def test_planner_allocation_failure_is_enomem(monkeypatch):
    s = mlev.Solver(W.config1(), device=-1)
    monkeypatch.setenv("MLEV_FAULT", "plan_alloc")
    with pytest.raises(mlev.MlevError) as e:
        s.workspace_bytes(mlev.default_opts())
    assert _code(e) == ENOMEM and "host allocation failed" in str(e.value)
    monkeypatch.delenv("MLEV_FAULT")
    assert s.workspace_bytes(mlev.default_opts()) > 0  # the context still works
    s.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -1.0])
def test_non_finite_or_negative_kappa_is_rejected(bad):
    p = W.kappa_coarse_batch(W.unit_square(4, 2, 3), batch=2, seed=1)
    p.kappa = p.kappa.copy()
    p.kappa[1, 2, 3] = bad
    with pytest.raises(mlev.MlevError) as e:
        mlev.Solver(p, device=-1)
    assert _code(e) == EINVAL and "kappa" in str(e.value)


def test_subdomain_without_cells_is_rejected():
    p = W.unit_square(4, 2, 3)
    p.cell_owner = np.where(p.cell_owner == 3, 2, p.cell_owner).astype(np.int32)  # D_2 takes D_3's cells
    with pytest.raises(mlev.MlevError) as e:
        mlev.Solver(p, device=-1)
    assert _code(e) == EINVAL and "owns no cell" in str(e.value)


def test_empty_closed_g_j_is_rejected():
    r = W.unit_square(4, 2, 3)
    r.delta = 2.0 * r.H  # every closed G_j would be empty
    with pytest.raises(mlev.MlevError) as e:
        mlev.Solver(r, device=-1)
    assert _code(e) == EINVAL


@pytest.mark.parametrize("field,value", [("vcycles", 0), ("refine_passes", 0), ("omega", 2.0), ("fused", 3),
                                         ("precision", 7), ("level1_tol", 0.0), ("rr_max_iter", 0)])
def test_invalid_options_are_einval(field, value):
    s = mlev.Solver(W.config1(), device=-1)
    o = mlev.default_opts()
    setattr(o, field, value)
    with pytest.raises(mlev.MlevError) as e:
        s.workspace_bytes(o)
    assert _code(e) == EINVAL and "invalid options" in str(e.value)
    s.close()


def test_call_order_violations_are_estate():
    import ctypes as C

    lib = mlev.load()
    h = C.c_void_p()
    assert lib.mlev_create(C.byref(h), -1) == 0
    owner = np.zeros((2, 2), np.int32)
    ov = np.zeros(1, np.int32)
    rc = lib.mlev_set_partition(h, 1, owner.ctypes.data_as(C.c_void_p), ov.ctypes.data_as(C.c_void_p), 0.25, 0)
    assert rc == ESTATE and b"domain" in lib.mlev_last_error(h)
    b = C.c_size_t()
    o = mlev.default_opts()
    assert lib.mlev_workspace_size(h, C.byref(o), C.byref(b)) == ESTATE
    assert lib.mlev_set_levels(h, 1) == EINVAL
    lib.mlev_destroy(h)


def test_planning_context_solve_is_estate():
    import ctypes as C

    s = mlev.Solver(W.config1(), device=-1)
    lam = np.zeros(1)
    rc = s.lib.mlev_solve(s.h, C.byref(mlev.default_opts()), C.c_void_p(256), 1 << 30, None,
                          lam.ctypes.data_as(C.c_void_p), None, None)
    assert rc == ESTATE and b"planning-only" in s.lib.mlev_last_error(s.h)
    s.close()


def test_glue_mode_other_than_the_paper_is_unsupported():
    import ctypes as C

    lib = mlev.load()
    h = C.c_void_p()
    assert lib.mlev_create(C.byref(h), -1) == 0
    cin = np.ones((4, 4), np.uint8)
    assert lib.mlev_set_domain(h, 4, 4, 0.0, 0.0, 0.25, cin.ctypes.data_as(C.c_void_p)) == 0
    owner = W.unit_square(4, 2, 3).cell_owner
    ov = np.ones(4, np.int32)
    rc = lib.mlev_set_partition(h, 4, owner.ctypes.data_as(C.c_void_p), ov.ctypes.data_as(C.c_void_p), 0.125, 1)
    assert rc == EUNSUPPORTED
    lib.mlev_destroy(h)


# ------------------------------------------------------------------ on the GPU (the solve runs)
@pytest.mark.gpu
def test_level1_iteration_cap_is_enoconv_and_context_recovers():
    s = mlev.Solver(W.config1())
    with pytest.raises(mlev.MlevError) as e:
        s.solve(mlev.default_opts(level1_max_iter=1, level1_tol=1e-14))
    assert _code(e) == ENOCONV and "cap" in str(e.value)
    lam, _, rep = s.solve(mlev.default_opts())
    assert rep["status_flags"] == 0 and abs(float(lam[0]) - 19.751102127489855) < 1e-7
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_rayleigh_ritz_iteration_cap_is_enoconv(prec):
    s = mlev.Solver(W.config1())
    with pytest.raises(mlev.MlevError) as e:
        s.solve(mlev.default_opts(precision=prec, rr_max_iter=1))
    assert _code(e) == ENOCONV and "cap" in str(e.value)
    s.close()


@pytest.mark.gpu
def test_workspace_too_small_is_enomem():
    import ctypes as C

    import torch

    s = mlev.Solver(W.config1())
    o = mlev.default_opts()
    need = s.workspace_bytes(o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    lam, _ = s.alloc_outputs()
    rc = s.lib.mlev_solve(s.h, C.byref(o), C.c_void_p(ws.data_ptr()), need - 256, None, C.c_void_p(lam.data_ptr()),
                          None, None)
    assert rc == ENOMEM and str(need).encode() in s.lib.mlev_last_error(s.h)
    rc = s.lib.mlev_solve(s.h, C.byref(o), C.c_void_p(ws.data_ptr() + 8), need, None, C.c_void_p(lam.data_ptr()),
                          None, None)
    assert rc == EINVAL and b"aligned" in s.lib.mlev_last_error(s.h)
    s.close()


@pytest.mark.gpu
def test_failed_table_copy_is_ecuda(monkeypatch):
    s = mlev.Solver(W.config1())
    monkeypatch.setenv("MLEV_FAULT", "h2d_copy")
    with pytest.raises(mlev.MlevError) as e:
        s.solve(mlev.default_opts())
    assert _code(e) == ECUDA and "injected" in str(e.value)
    monkeypatch.delenv("MLEV_FAULT")
    lam, _, rep = s.solve(mlev.default_opts())  # the tables are copied again on the next call
    assert rep["status_flags"] == 0 and abs(float(lam[0]) - 19.751102127489855) < 1e-7
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_non_finite_coefficient_on_the_device_is_enoconv(monkeypatch, prec):
    p = W.kappa_coarse_batch(W.unit_square(8, 2, 3), batch=2, seed=4)
    s = mlev.Solver(p)
    monkeypatch.setenv("MLEV_FAULT", "kappa_nan")
    with pytest.raises(mlev.MlevError) as e:
        s.solve(mlev.default_opts(precision=prec))
    assert _code(e) == ENOCONV and "status flags" in str(e.value)
    monkeypatch.delenv("MLEV_FAULT")
    s2 = mlev.Solver(p)  # a fresh context uploads clean values
    lam, _, rep = s2.solve(mlev.default_opts(precision=prec))
    assert rep["status_flags"] == 0 and np.all(np.isfinite(lam.cpu().numpy()))
    s.close()
    s2.close()
