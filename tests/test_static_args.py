"""The binding of lpdf_pdf_step_static rejects buffers of the wrong dtype, shape, layout or device
before any launch (the library gets bare pointers and cannot size them). CPU tensors only."""
import pytest

torch = pytest.importorskip("torch")

from paper_1006_0549_gb300 import lpdf, workloads as wl  # noqa: E402


def _good(n=10, n_nodes=7, ns=2, device="cpu"):
    f = lambda *s: torch.zeros(s, dtype=torch.float32, device=device)
    st = {k: f(n) for k in ("x", "y", "u", "v", "w", "omega")}
    st["psi"] = f(ns, n)
    st["elem"] = torch.zeros(n, dtype=torch.int32, device=device)
    st["pid"] = torch.zeros(n, dtype=torch.int32, device=device)
    F = f(n_nodes, wl.n_fields_padded(ns))
    M = torch.zeros((n_nodes, 11 + 2 * ns), dtype=torch.float64, device=device)
    return st, F, M


def _raises(match, n_nodes, ns, st, F, M):
    with pytest.raises(ValueError, match=match):
        lpdf.check_static_args(n_nodes, ns, st, F, M)


def test_cpu_buffers_are_rejected_for_the_device_only():
    st, F, M = _good()
    _raises("CUDA device", 7, 2, st, F, M)


@pytest.mark.parametrize("key", ["x", "omega", "psi", "elem", "pid"])
def test_wrong_dtype(key):
    st, F, M = _good()
    st[key] = st[key].to(torch.float64)
    _raises("must be", 7, 2, st, F, M)


def test_wrong_shapes():
    st, F, M = _good()
    st["u"] = torch.zeros(9, dtype=torch.float32)
    _raises("shape", 7, 2, st, F, M)
    st, F, M = _good()
    st["psi"] = torch.zeros((3, 10), dtype=torch.float32)      # ns rows, not 3
    _raises("shape", 7, 2, st, F, M)
    st, F, M = _good()
    _raises("node_fields must have shape", 8, 2, st, F, M)     # n_nodes of another mesh
    st, F, M = _good()
    M = torch.zeros((7, 11), dtype=torch.float64)
    _raises("moments must have shape", 7, 2, st, F, M)
    st, F, M = _good()
    _raises("ns must be", 7, 5, st, F, M)


def test_non_contiguous_and_missing():
    st, F, M = _good()
    st["psi"] = torch.zeros((10, 2), dtype=torch.float32).t()
    _raises("contiguous", 7, 2, st, F, M)
    st, F, M = _good()
    del st["pid"]
    _raises("lacks", 7, 2, st, F, M)


def test_meta_tensors_pass_the_layout_checks():
    st, F, M = _good(device="meta")
    _raises("CUDA device", 7, 2, st, F, M)
