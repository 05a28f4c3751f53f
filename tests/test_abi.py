"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/afc.h declares, and rejects bad arguments before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "afc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(afc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("afc_create_structured", "afc_create_from_elements", "afc_set_coefficients", "afc_set_dirichlet",
                 "afc_assemble", "afc_step", "afc_solve_stationary", "afc_destroy", "afc_export_csr"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2110_15676_gb300 import afc
    lib = C.CDLL(afc.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(afc.EXPORTED) == set(_declared())


def test_default_options_and_status_strings():
    from paper_2110_15676_gb300 import afc
    o = afc.default_opts()
    assert o.fp_tol == 1e-10 and o.ksp_atol == 1e-12 and o.gmres_restart == 20 and o.prelimit == 1
    assert afc.afc_status_str(afc.AFC_OK) == b"ok"
    assert b"invalid" in afc.afc_status_str(afc.AFC_E_INVALID)


def test_invalid_meshes_rejected_on_host():
    from paper_2110_15676_gb300 import afc
    with pytest.raises(afc.AfcError) as e:
        afc.Problem.structured("p1", (1, 4, 4))
    assert e.value.status == afc.AFC_E_INVALID
    with pytest.raises(afc.AfcError):
        afc.Problem.structured("q1", 4, lo=(0, 0, 0), hi=(1, 0, 1))
    # out-of-range connectivity
    xyz = np.zeros((4, 3))
    with pytest.raises(afc.AfcError) as e:
        afc.Problem.from_elements("p1", xyz, np.array([[0, 1, 2, 7]]))
    assert e.value.status == afc.AFC_E_INVALID
    # too many distinct column offsets for the diagonal-offset storage
    rng = np.random.default_rng(0)
    n = 200
    conn = np.stack([rng.choice(n, 4, replace=False) for _ in range(60)])
    with pytest.raises(afc.AfcError) as e:
        afc.Problem.from_elements("p1", rng.uniform(size=(n, 3)), conn)
    assert "offsets" in str(e.value)


def test_grid_wait_selftest_rejects_bad_limits_on_host():
    from paper_2110_15676_gb300 import afc
    obs = C.c_int(-1)
    for bad in (0.0, -1.0, 4001.0, float("nan")):
        assert afc.afc_selftest_grid_wait(0, bad, C.byref(obs), None) == afc.AFC_E_INVALID
    assert afc.afc_selftest_grid_wait(0, 10.0, None, None) == afc.AFC_E_INVALID
    assert obs.value == -1


def test_device_vector_checks_reject_bad_tensors_before_any_call():
    """afc_mc_limited_sum_noalloc takes raw device pointers, so the binding checks
    each tensor (CUDA, float64, contiguous, N elements, the problem's device) and
    raises AFC_E_INVALID before the library could read or write past its end."""
    torch = pytest.importorskip("torch")
    from paper_2110_15676_gb300 import afc

    class FakeCuda:   # stands in for a CUDA tensor on this machine without a GPU
        def __init__(self, n=10, dtype=torch.float64, contiguous=True, index=0):
            self.is_cuda, self.dtype, self._c, self._n = True, dtype, contiguous, n
            self.device = type("dev", (), {"index": index})()

        def data_ptr(self):
            return 0

        def is_contiguous(self):
            return self._c

        def numel(self):
            return self._n

    afc.check_device_vector(FakeCuda(), 10, 0, "u", "t")     # accepted
    cases = [(torch.zeros(10, dtype=torch.float64), "CUDA"), (FakeCuda(dtype=torch.float32), "dtype"),
             (FakeCuda(contiguous=False), "contiguous"), (FakeCuda(n=9), "elements"),
             (FakeCuda(index=1), "cuda:1"), (np.zeros(10), "tensor")]
    for t, why in cases:
        with pytest.raises(afc.AfcError) as e:
            afc.check_device_vector(t, 10, 0, "u", "afc_mc_limited_sum_noalloc")
        assert e.value.status == afc.AFC_E_INVALID and why in str(e.value)
