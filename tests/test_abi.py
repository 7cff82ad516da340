"""The C-ABI library builds, loads and exports every symbol include/lsp.h declares (no GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("lsp_plan_create", "lsp_set_potential", "lsp_set_state", "lsp_strang_steps",
              "lsp_get_state", "lsp_plan_destroy", "lsp_strerror", "lsp_batch_create",
              "lsp_batch_steps", "lsp_adjoint", "lsp_lattice_points", "lsp_index_table"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1808_06357_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_1808_06357_gb300 as lsp
    assert lsp.strerror(0) == "ok"
    assert "canonical" in lsp.strerror(-2)
    assert lsp.strerror(12345) == "unknown status"


def test_plan_create_fails_loudly_without_gpu():
    """With no usable device the binding raises; nothing falls back to the CPU."""
    import numpy as np
    import pytest
    import torch
    import paper_1808_06357_gb300 as lsp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lsp.LspError) as e:
        lsp.Plan(np.array([1, 5]), (64,), 0.1)
    assert e.value.code == -6


def test_binding_resolves_conjugate_views():
    """A lazily conjugated torch view is materialised before its pointer is passed; as an
    output it is refused (its memory does not hold the values it represents)."""
    import numpy as np
    import pytest
    import torch
    from paper_1808_06357_gb300 import _binding as B
    x = torch.tensor([1 + 2j, 3 - 4j], dtype=torch.complex128)
    cx = torch.conj(x)
    assert cx.is_conj()
    ptr, dev = B._buf(cx)
    got = np.ctypeslib.as_array((ctypes.c_double * 4).from_address(ptr.value))
    assert np.array_equal(got, [1.0, -2.0, 3.0, 4.0]) and dev == 0
    with pytest.raises(ValueError):
        B._buf(cx, output=True)


def test_cbc_argument_checks_without_gpu():
    """lsp_cbc_reconstructing rejects bad shapes and moduli before touching a device, and reports
    a missing device as CUDA (never a CPU fallback)."""
    import numpy as np
    import pytest
    import torch
    import paper_1808_06357_gb300 as lsp
    I = np.array([[0, 0], [1, 0], [0, 1]])
    cand = np.array([[[3]]])
    with pytest.raises(lsp.LspError) as e:
        lsp.cbc_reconstructing(I, (8, 4, 2), np.zeros((1, 1, 3), dtype=np.int64))   # rank 3
    assert e.value.code == -1
    with pytest.raises(lsp.LspError) as e:
        lsp.cbc_reconstructing(I, 0, cand)                                           # modulus 0
    assert e.value.code == -1
    with pytest.raises(lsp.LspError) as e:
        lsp.cbc_reconstructing(I, (1 << 20, 1 << 12), np.zeros((1, 1, 2), dtype=np.int64))  # 2^32 bins
    assert e.value.code == -1
    if not torch.cuda.is_available():
        with pytest.raises(lsp.LspError) as e:
            lsp.cbc_reconstructing(I, 8, cand)
        assert e.value.code == -6


def test_noalloc_binding_refuses_unchecked_buffers():
    """The allocation-free entry point takes raw pointers: the binding refuses host
    arrays, wrong dtypes and short buffers before any call reaches the library."""
    import numpy as np
    import pytest
    import torch
    import paper_1808_06357_gb300 as lsp
    u = np.zeros(16, dtype=np.complex64)
    v = np.zeros(16)
    nrm = np.zeros(16, dtype=np.int32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lsp.strang_steps_noalloc(u, v, nrm, 0.1, 1e-3, 1)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lsp.strang_steps_noalloc(torch.zeros(16, dtype=torch.complex64), torch.zeros(16, dtype=torch.float64),
                                 torch.zeros(16, dtype=torch.int32), 0.1, 1e-3, 1)


def test_plan_create_rank_checks_before_any_device_call():
    """Rank and canonical-form checks (Def. 1, Sec. 2.5) come before the device is touched, so
    they answer the same with or without a GPU: r <= 4, and n_{i+1} divides n_i."""
    import numpy as np
    import pytest
    import paper_1808_06357_gb300 as lsp
    with pytest.raises(lsp.LspError) as e:                  # rank 5
        lsp.Plan(np.eye(5, dtype=np.int64), (2, 2, 2, 2, 2), 0.1)
    assert e.value.code == -1
    with pytest.raises(lsp.LspError) as e:                  # 3 does not divide 8
        lsp.Plan(np.eye(3, dtype=np.int64), (8, 3, 3), 0.1)
    assert e.value.code == -2
