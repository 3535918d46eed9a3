"""Shared test helpers: uniform node fields and state builders (inputs only)."""
import numpy as np

from paper_1006_0549_gb300 import workloads as wl


def uniform_fields(mesh, ns, **vals):
    """Node fields equal at every node; keyword names are the F_* suffixes in lower case."""
    nfp = wl.n_fields_padded(ns)
    F = np.zeros((mesh.n_nodes, nfp), dtype=np.float32)
    names = {
        "u": wl.F_U, "v": wl.F_V, "w": wl.F_W, "dudx": wl.F_DUDX, "dudy": wl.F_DUDY,
        "dvdx": wl.F_DVDX, "dvdy": wl.F_DVDY, "dwdx": wl.F_DWDX, "dwdy": wl.F_DWDY,
        "lapu": wl.F_LAPU, "lapv": wl.F_LAPV, "lapw": wl.F_LAPW, "dpdx": wl.F_DPDX, "dpdy": wl.F_DPDY,
        "g11": wl.F_G11, "g12": wl.F_G12, "g21": wl.F_G21, "g22": wl.F_G22, "g33": wl.F_G33,
        "c0eps": wl.F_C0EPS, "omega": wl.F_OMEGA, "somega": wl.F_SOMEGA,
    }
    for k, v in vals.items():
        if k.startswith("phi"):
            F[:, wl.F_PHI0 + int(k[3:])] = v
        else:
            F[:, names[k]] = v
    return F


def state_from(res, elem, pid, ns):
    """workloads.State (FP32) from an oracle result dict."""
    return wl.State(*(np.asarray(res[k], dtype=np.float32) for k in ("x", "y", "u", "v", "w", "omega")),
                    np.asarray(res["psi"], dtype=np.float32).reshape(ns, -1),
                    np.asarray(elem, dtype=np.int32), np.asarray(pid, dtype=np.uint32))
