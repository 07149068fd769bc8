"""The C-ABI library builds for sm_103a, loads on a host without a GPU, and
exports every entry point include/swr.h declares.  No compute calls."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "swr.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(swr_\w+)\s*\(", hdr, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libswr():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1503_02564_gb300 import build_ext
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("swr_plan", "swr_build_interface", "swr_solve", "swr_adjoint", "swr_destroy",
              "swr_status_string", "swr_apply_R", "swr_apply_interface", "swr_get_interface",
              "swr_apply_precond", "swr_misfit"):
        assert f in names, f


def test_library_exports_every_declared_symbol(libswr):
    for name in _declared():
        assert hasattr(libswr, name), name


def test_status_strings_without_gpu(libswr):
    libswr.swr_status_string.restype = ctypes.c_char_p
    libswr.swr_status_string.argtypes = [ctypes.c_int]
    for code in range(10):
        assert libswr.swr_status_string(code).startswith(b"SWR_")


def test_plan_rejects_bad_arguments_without_touching_the_device(libswr):
    from paper_1503_02564_gb300 import swr
    h = ctypes.c_void_p()
    assert libswr.swr_plan(None, ctypes.byref(h), None) == swr.SWR_ERR_ARG
    d = swr.swr_desc()
    d.nx = 2                      # too few nodes
    assert libswr.swr_plan(ctypes.byref(d), ctypes.byref(h), None) == swr.SWR_ERR_ARG
    assert not h.value


def _desc(**kw):
    from paper_1503_02564_gb300 import swr
    d = swr.swr_desc()
    d.nx, d.a0, d.b0, d.nt, d.dt, d.nsub = 101, -1.0, 1.0, 10, 1e-3, 4
    d.vkind, d.tc, d.tc_re, d.tc_im = swr.SWR_V_STATIC, swr.SWR_TC_ROBIN, 1.58, -1.58
    d.solver, d.precond, d.pc_sweeps = swr.SWR_SOLVER_GMRES, swr.SWR_PC_NONE, -1
    for k, v in kw.items():
        setattr(d, k, v)
    return d


def _rejects(libswr, descs, want, off=None):
    """Every case below is refused during validation, before any device call."""
    h = ctypes.c_void_p()
    arr = (type(descs[0]) * len(descs))(*descs)
    if len(descs) == 1:
        rc = libswr.swr_plan(ctypes.byref(arr[0]), ctypes.byref(h), None)
    else:
        rc = libswr.swr_plan_batch(arr, len(descs), ctypes.byref(h), None)
    assert rc == want, (rc, want)
    assert not h.value


def _bad_cases():
    from paper_1503_02564_gb300 import swr as S
    A, U = S.SWR_ERR_ARG, S.SWR_ERR_UNSUPPORTED
    return [
        ("no time steps", dict(nt=0), A),
        ("non-positive dt", dict(dt=0.0), A),
        ("one subdomain", dict(nsub=1), A),
        ("empty interval", dict(b0=-1.0), A),
        ("potential kind", dict(vkind=3), A),
        ("transmission condition", dict(tc=6), A),
        ("solver", dict(solver=5), A),
        ("preconditioner", dict(precond=4), A),
        ("S_0^3 with V(t,x)", dict(tc=S.SWR_TC_S03, vkind=S.SWR_V_TIME), U),
        ("S_1^4 with the mean-potential operator",
         dict(tc=S.SWR_TC_S14, precond=S.SWR_PC_MEAN_POTENTIAL), U),
        ("BiCGStab, nonlinear", dict(solver=S.SWR_SOLVER_BICGSTAB, vkind=S.SWR_V_NONLINEAR), A),
        ("direct causal solve, V(t,x)", dict(solver=S.SWR_SOLVER_CAUSAL, vkind=S.SWR_V_TIME), A),
        ("GMRES, nonlinear", dict(solver=S.SWR_SOLVER_GMRES, vkind=S.SWR_V_NONLINEAR), A),
        ("fixed point, V(t,x)", dict(solver=S.SWR_SOLVER_FIXED_POINT, vkind=S.SWR_V_TIME), A),
        ("causal preconditioner, V(t,x)", dict(precond=S.SWR_PC_CAUSAL, vkind=S.SWR_V_TIME), A),
        ("V(t,x) table beyond 2^31 entries",
         dict(vkind=S.SWR_V_TIME, nx=2_000_001, nt=1100, solver=S.SWR_SOLVER_GMRES), A),
        ("flux blocks beyond 32-bit offsets", dict(nx=400_001, nsub=100_000, nt=4000), A),
    ]


@pytest.mark.parametrize("case", range(17))
def test_plan_validation_refuses_unsupported_descriptions(libswr, case):
    name, kw, want = _bad_cases()[case]
    _rejects(libswr, [_desc(**kw)], want)


@pytest.mark.parametrize("off", [[1, 30, 60, 100], [0, 30, 60, 99], [0, 30, 31, 100],
                                 [0, 60, 30, 100]])
def test_plan_validation_refuses_bad_partitions(libswr, off):
    """node_off must start at 0, end at nx - 1 and give every subdomain >= 2 elements."""
    arr = (ctypes.c_int32 * len(off))(*off)
    d = _desc(nsub=len(off) - 1)
    d.node_off = ctypes.cast(arr, type(d.node_off))
    _rejects(libswr, [d], 1)


def test_batch_validation_refuses_mismatched_instances(libswr):
    """A batch shares dt, the transmission condition and the solver settings; time-dependent
    potentials are not batched; an empty batch is refused."""
    from paper_1503_02564_gb300 import swr as S
    _rejects(libswr, [_desc(), _desc(dt=2e-3)], S.SWR_ERR_ARG)
    _rejects(libswr, [_desc(), _desc(tc_re=1.0)], S.SWR_ERR_ARG)
    _rejects(libswr, [_desc(), _desc(nx=201, b0=3.0, restart=20)], S.SWR_ERR_ARG)
    _rejects(libswr, [_desc(vkind=S.SWR_V_TIME), _desc(vkind=S.SWR_V_TIME)],
             S.SWR_ERR_UNSUPPORTED)
    h = ctypes.c_void_p()
    d = _desc()
    assert libswr.swr_plan_batch(ctypes.byref(d), 0, ctypes.byref(h), None) == S.SWR_ERR_ARG


def test_binding_has_no_cpu_path(monkeypatch, tmp_path):
    """The binding refuses host tensors (the compute path is the CUDA library only) and
    raises when the library has not been built, instead of falling back to anything."""
    import torch
    from paper_1503_02564_gb300 import swr
    with pytest.raises(TypeError):
        swr._ptr(torch.zeros(4, dtype=torch.float64), torch.float64, 4, "V")
    monkeypatch.setattr(swr, "_lib", None)
    monkeypatch.setattr(swr, "LIB_PATH", str(tmp_path / "libswr.so"))
    with pytest.raises(RuntimeError, match="not built"):
        swr.lib()
