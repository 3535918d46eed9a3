"""Writes the oracle regression fixtures of this folder.

The paper prints no worked numerical example: no table of values, no constants of the model, no
sizes of its runs beyond the Reynolds numbers of its two testcases (Section "Two testcases":
Re_tau = 1080 for the channel, Re = 4000 for the cavity), which are configuration values, not
results. So nothing here is a printed value of the paper. These fixtures freeze what the FP64
oracle computes on tiny seeded inputs (including a step on a channel with a curved wall), so that any later change of its arithmetic shows up as a
failing test and has to be justified by the passage it follows. This script calls only the oracle
and the seeded input generators (which hold none of the method's arithmetic).

    python tests/golden/make_golden.py      # rewrites oracle_fixtures.txt
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle                                               # noqa: E402
from paper_1006_0549_gb300 import workloads as wl           # noqa: E402

OUT = os.path.join(HERE, "oracle_fixtures.txt")

PHILOX_CASES = [((0, 0, 0, 0), (0, 0)), ((1, 2, 3, 4), (5, 6)),
                ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF)), ((12345, 7, 0, 1 << 16), (1006054901, 0))]
NORMAL_CASES = [(1006054901, 0, 0, 0), (1006054901, 123456, 17, 0), (42, 7, 1 << 33, 1)]


def step_case():
    """One step of a tiny channel (6 x 4 cells, 3 particles per element, one scalar, a source)."""
    mesh = wl.channel_mesh(6, 4, 11)
    om = oracle.OracleMesh(mesh)
    st = wl.synthetic_state(mesh, 3, 1, seed=21)
    F = wl.synthetic_node_fields(mesh, 1, seed=22)
    p = oracle.make_params(nu=1.0 / 180.0, dt=1e-3, seed=23, ns=1, sources=[(0.25, 0.67, 0.3, 0)])
    res, elem, _, lost = oracle.pdf_step(om, p, F, st, 5)
    S, _ = oracle.moments(om, 1, res["x"], res["y"], res["u"], res["v"], res["w"], res["omega"], res["psi"], elem)
    return res, elem, lost, S


def walls_case():
    """One step on a small channel with a curved bottom wall (12 x 6 cells), fast wall-normal
    motion so that particles meet the walls and the periodic seam: walls mirrored in the walk."""
    mesh = wl.bump_channel_mesh(12, 6, 7, amp=0.3)
    om = oracle.OracleMesh(mesh)
    st = wl.synthetic_state(mesh, 3, 1, seed=31)
    st.u = (st.u * 4.0).astype(np.float32)
    st.v = (st.v * 20.0).astype(np.float32)
    F = wl.synthetic_node_fields(mesh, 1, seed=32)
    p = oracle.make_params(nu=1.0 / 180.0, dt=1e-3, seed=33, ns=1)
    res, elem, aux, lost = oracle.pdf_step(om, p, F, st, 2, locate_mode=2)
    return res, elem, aux, lost


def lines():
    out = []
    for ctr, key in PHILOX_CASES:
        w = oracle.philox4x32_10(ctr, key)
        out.append("philox %s %s : %s" % (" ".join("%08x" % c for c in ctr), " ".join("%08x" % k for k in key),
                                           " ".join("%08x" % int(x) for x in w)))
    for seed, pid, step, tag in NORMAL_CASES:
        z = oracle.normals6(seed, pid, step, tag)
        out.append("normals6 %d %d %d %d : %s" % (seed, pid, step, tag, " ".join("%.17g" % v for v in z)))
    res, elem, lost, S = step_case()
    out.append("step lost : %d" % lost)
    for k in ("x", "y", "u", "v", "w", "omega"):
        out.append("step %s : %s" % (k, " ".join("%.17g" % v for v in res[k])))
    out.append("step psi0 : %s" % " ".join("%.17g" % v for v in res["psi"][0]))
    out.append("step elem : %s" % " ".join("%d" % e for e in elem))
    out.append("moments : %s" % " ".join("%.17g" % v for v in S.ravel()))
    res, elem, aux, lost = walls_case()
    out.append("walls lost : %d" % lost)
    for k in ("x", "y", "u", "v"):
        out.append("walls %s : %s" % (k, " ".join("%.17g" % v for v in res[k])))
    out.append("walls elem : %s" % " ".join("%d" % e for e in elem))
    out.append("walls mirrorings : %s" % " ".join("%d" % int(v) for v in aux[:, 2]))
    return out


if __name__ == "__main__":
    with open(OUT, "w") as f:
        f.write("# written by tests/golden/make_golden.py from the FP64 oracle; see that script's docstring\n")
        f.write("\n".join(lines()) + "\n")
    print("wrote", OUT)
