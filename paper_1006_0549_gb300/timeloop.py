"""The coupled time loop of the method through the C-ABI: particle step (lpdf_pdf_step), gridpoint
statistics (lpdf_grid_statistics), gridpoint solve for the next step's node fields
(lpdf_elliptic_relax_solve, or the learned surrogate through lpdf_surrogate_relax_solve).
Introduction, items i-iii: statistics are extracted on the grid, Eulerian quantities are solved on
it, and the particles are advanced with them. Orchestration only: every computation is a library call.
"""
from __future__ import annotations

import numpy as np

from . import lpdf
from . import workloads as wl


class TimeLoop:
    """One ensemble on one mesh, with its statistics and node-field buffers on the device."""

    def __init__(self, wk: wl.Workload, params: lpdf.Params, tol: float = 1e-8, maxit: int = 20000,
                 init_seed: int = 5, capacity: int | None = None):
        import torch
        self.torch = torch
        self.wk = wk
        self.mesh = lpdf.Mesh(wk.mesh)
        self.params = params
        self.tol, self.maxit = tol, maxit
        N = wk.mesh.n_nodes
        self.N = N
        self.nq = 11 + 2 * wk.ns
        self.nfp = wl.n_fields_padded(wk.ns)
        cap = capacity or wk.n_particles + 1024
        self.ctx = lpdf.Context(self.mesh, params, cap)
        self.ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda(), m_erlang=4)
        self.S = torch.zeros((N, self.nq), dtype=torch.float64, device="cuda")
        self.F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=init_seed)).cuda()
        self.step_no = 0
        # the first step runs on seeded synthetic node fields; its statistics start the loop
        self.advance()

    def advance(self):
        """One particle step with the current node fields, then the statistics of the new state."""
        self.step_no += 1
        self.ctx.pdf_step(self.F, self.step_no)
        self.ctx.grid_statistics(self.S, raw=False)

    def solve_plain(self):
        return self.mesh.elliptic_relax_solve(self.params, self.S, self.F, self.tol, self.maxit)

    def solve_surrogate(self, net: lpdf.MLP):
        return self.mesh.surrogate_relax_solve(net, self.params, self.S, self.F, self.tol, self.maxit)

    def features(self, with_targets: bool = True):
        """Network inputs (and targets from the current node fields) of the current statistics."""
        torch = self.torch
        f = torch.empty((self.N, lpdf.MLP_IN), dtype=torch.float32, device="cuda")
        t = torch.empty((self.N, lpdf.MLP_OUT), dtype=torch.float32, device="cuda") if with_targets else None
        self.mesh.surrogate_features(self.params, self.S, f, self.F if with_targets else None, t)
        return f, t

    def snapshot(self):
        return self.ctx.get_state(), self.S.clone(), self.F.clone(), self.step_no

    def restore(self, snap, params: lpdf.Params | None = None):
        st, S, F, n = snap
        self.ctx.set_state(st)
        self.S.copy_(S)
        self.F.copy_(F)
        self.step_no = n
        if params is not None:
            self.params = params
            self.ctx.set_params(params)


def collect_training_data(loop: TimeLoop, steps: int):
    """`steps` plain steps; returns the network inputs and targets of every solve (device)."""
    torch = loop.torch
    feats, tgts = [], []
    for _ in range(steps):
        loop.solve_plain()
        f, t = loop.features(True)
        feats.append(f)
        tgts.append(t)
        loop.advance()
    return torch.cat(feats), torch.cat(tgts)


def train_surrogate(feat, tgt, seed: int = 7, batch: int = 1024,
                    schedule=((1e-3, 4000), (3e-4, 3000), (1e-4, 3000))):
    """A network trained on (feat, tgt) with Adam, in shuffled minibatches (a seeded permutation),
    with a stepwise decaying learning rate. Returns (network, loss history)."""
    import torch
    B = feat.shape[0]
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(B)).to(feat.device)
    feat, tgt = feat[perm].contiguous(), tgt[perm].contiguous()
    net = lpdf.MLP(batch)
    net.set_params(wl.mlp_init_params(seed))
    net.fit_norm(feat, tgt)
    n = B // batch * batch
    hist = [net.train(feat[:n], tgt[:n], batch=batch, steps=k, lr=lr) for lr, k in schedule]
    return net, np.concatenate(hist)


def relative_difference(a, b, cols):
    """|a - b| / |b| (Frobenius) over the given statistics columns."""
    a = np.asarray(a)[:, cols]
    b = np.asarray(b)[:, cols]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_surrogate(loop: TimeLoop, net: lpdf.MLP, steps: int, train_feat=None, train_tgt=None, retrain_steps: int = 0,
                  retrain_lr: float = 3e-4, batch: int = 1024, seed: int = 17):
    """`steps` steps with the surrogate solve. With retrain_steps > 0 the network keeps learning:
    a failed check (its plain fields are the step's fields) adds that step's inputs and targets to
    a set of new rows, the network takes retrain_steps more Adam steps on the new rows mixed with
    as many rows drawn from the earlier training data (train_feat, train_tgt), and the next solve
    checks again. Returns a dict of what happened (per-step solve times, whether the plain solve
    ran, check errors, calls on the network, retrainings)."""
    import torch
    rng = np.random.default_rng(seed)
    new_f, new_t = [], []
    times, errs, used, retrains = [], [], 0, 0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        checked, err, used_plain, _ = loop.solve_surrogate(net)
        e1.record()
        torch.cuda.synchronize()
        times.append((e0.elapsed_time(e1), used_plain))
        if checked:
            errs.append(err)
        used += 0 if used_plain else 1
        if checked and retrain_steps > 0 and err > net.threshold:
            f, t = loop.features(True)
            new_f.append(f)
            new_t.append(t)
            Fn, Tn = torch.cat(new_f), torch.cat(new_t)
            if train_feat is not None:
                pick = torch.from_numpy(rng.integers(0, train_feat.shape[0], Fn.shape[0])).to(Fn.device)
                Fn, Tn = torch.cat([Fn, train_feat[pick]]), torch.cat([Tn, train_tgt[pick]])
            perm = torch.from_numpy(rng.permutation(Fn.shape[0])).to(Fn.device)
            n = max(batch, Fn.shape[0] // batch * batch)
            b = min(batch, Fn.shape[0])
            net.train(Fn[perm][:n].contiguous(), Tn[perm][:n].contiguous(), batch=b, steps=retrain_steps,
                      lr=retrain_lr)
            net.request_check()
            retrains += 1
        loop.advance()
    return {"times": times, "check_errors": errs, "network_used_on": used, "retrains": retrains}


def run_coupled(wk: wl.Workload, params: lpdf.Params, state: dict, fields0, steps: int, record=(),
                tol: float = 1e-12, maxit: int = 20000, step0: int = 1, timing: bool = False):
    """The plain coupled loop from a given state: for n = 1..steps, lpdf_pdf_step with the current
    node fields (Philox step number step0 + n - 1), lpdf_grid_statistics (means and central
    moments), and, before the next step, lpdf_elliptic_relax_solve for the next node fields.
    `state` is a dict of device tensors for lpdf_set_state, fields0 the first step's node fields
    (device). Returns (statistics at the steps in `record` as {n: host array}, per-step device
    times {"step_ms", "solve_ms"} when timing, the final status)."""
    import torch
    gm = lpdf.Mesh(wk.mesh)
    n = int(state["x"].shape[0])
    ctx = lpdf.Context(gm, params, n)
    ctx.set_state(state)
    F = fields0.clone()
    S = torch.zeros((wk.mesh.n_nodes, 11 + 2 * params.ns), dtype=torch.float64, device="cuda")
    out, step_ms, solve_ms = {}, [], []
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for k in range(1, steps + 1):
        e0, e1, e2 = ev(), ev(), ev()
        e0.record()
        ctx.pdf_step(F, step0 + k - 1)
        ctx.grid_statistics(S, raw=False)
        e1.record()
        if k in record:
            out[k] = S.cpu().numpy()
        if k < steps:
            gm.elliptic_relax_solve(params, S, F, tol, maxit)
        e2.record()
        if timing:
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            solve_ms.append(e1.elapsed_time(e2))
    torch.cuda.synchronize()
    rc, status = ctx.status(raise_on_error=False)
    return out, {"step_ms": step_ms, "solve_ms": solve_ms}, (rc, status)
