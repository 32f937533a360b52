"""Learned coarse-grid closure: training pairs generated by the solver, training
and evaluation.

A pair is one sound-wave or normal-shock instance solved on a fine grid
(4096 cells) and on an 8x coarser grid (512 cells) over the same domain and the
same physical times (the coarse time step is 8x the fine one).  At each of 8
snapshots the network input is the coarse fields (rho, u, T, q, Pxx) plus two
constant channels (eta0 and log10 of the mean free path over the cell size),
and the target is the fine fields averaged 8:1 onto the coarse cells minus the
coarse fields.  The network corrects coarse fields after the fact; the solver
state is not modified, and the plain fine-grid solve remains the reference for
its error.

Solves, field restriction, training and inference run in the library's kernels
(libqlbm.so); this module only moves device tensors between those calls.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs
from . import qlbm as q

NF, NC = 4096, 512
FIELDS = ("rho", "u", "T", "q", "Pxx")


def pair_specs(n: int, seed0: int):
    """Seeded pair parameters: alternating sound waves (Q = 16) and shocks (Q = 32),
    E_l ~ U[0.02, 0.3], Mach ~ U[1.2, 3] (upstream temperature inputs.SHOCK_T_UPSTREAM, as in
    the batched workload)."""
    out = []
    for j in range(n):
        rng = np.random.default_rng(seed0 + j)
        El = float(rng.uniform(0.02, 0.3))
        mach = float(rng.uniform(1.2, 3.0))
        if j % 2 == 0:
            out.append(dict(kind="sound", Q=16, denseness=El, kn=0.1, length=1.0,
                            prm=(1.0, 1.0, float(rng.uniform(5e-3, 5e-2)))))
        else:
            out.append(dict(kind="shock", Q=32, denseness=El, kn=1.0 / 128.0, length=128.0,
                            prm=(1.0, inputs.SHOCK_T_UPSTREAM, mach, 4.0)))
    return out


def _instances(specs, nx, dt_of):
    keep, insts = [], []
    for s in specs:
        sound = s["kind"] == "sound"
        insts.append(q.make_instance(s["Q"], nx, s["length"], dt_of(s), s["denseness"], s["kn"],
                                     bc=q.QL_BC_PERIODIC if sound else q.QL_BC_FIXED,
                                     init_kind=q.QL_INIT_SOUND if sound else q.QL_INIT_SHOCK, prm=s["prm"],
                                     keep=keep))
    return insts, keep


def _fine_dt(s):
    p, _ = q.ql_velocity_set(s["Q"])
    return inputs.cfl_dt(s["length"] / NF, float(np.abs(p).max()))


def const_channels(specs, device):
    """Per pair: the constant input channels (eta0, log10 of the mean free path over the coarse cell
    size) [N][2] and the padding kind (1 periodic, 0 replicated ends) [N], as device tensors."""
    import torch
    consts = torch.tensor([[q.ql_eta_of_denseness(s["denseness"]), math.log10(s["kn"] * s["length"] / (s["length"] / NC))]
                           for s in specs], dtype=torch.float32, device=device)
    periodic = torch.tensor([1 if s["kind"] == "sound" else 0 for s in specs], dtype=torch.int32, device=device)
    return consts, periodic


def generate(specs, fine_steps: int, snapshots: int = 8, precision=q.QL_FP32, return_fine_state=False):
    """Runs the fine and coarse solves of every pair; returns device tensors
    x [N snapshots][NC][7], y [N][NC][5], periodic [N] and the coarse fields."""
    import torch
    assert fine_steps % (8 * snapshots) == 0
    dev = torch.device("cuda", torch.cuda.current_device())
    fine_i, k1 = _instances(specs, NF, _fine_dt)
    coarse_i, k2 = _instances(specs, NC, lambda s: 8.0 * _fine_dt(s))
    fb = q.Batch(fine_i, precision=precision)
    cb = q.Batch(coarse_i, precision=precision)
    n = len(specs)
    consts, periodic = const_channels(specs, dev)
    ff = torch.empty(n * 5 * NC, dtype=torch.float64, device=dev)
    cf = torch.empty(n * 5 * NC, dtype=torch.float64, device=dev)
    xs, ys, ps, coarse = [], [], [], []
    cur = torch.cuda.current_stream()
    for s in range(snapshots):
        # the field buffers are reused: the solver streams wait for the last snapshot's copies
        fb._stream.wait_stream(cur)
        cb._stream.wait_stream(cur)
        fb.run(fine_steps // snapshots)
        cb.run(fine_steps // snapshots // 8)
        fb.fields(NC, ff)
        cb.fields(NC, cf)
        cur.wait_stream(fb._stream)
        cur.wait_stream(cb._stream)
        F = ff.view(n, 5, NC).permute(0, 2, 1).float()
        Cc = cf.view(n, 5, NC).permute(0, 2, 1).float()
        xs.append(torch.cat([Cc, consts[:, None, :].expand(n, NC, 2)], dim=2))
        ys.append(F - Cc)
        ps.append(periodic)
        coarse.append(Cc)
    fb.sync()
    cb.sync()
    fb.close()
    cb.close()
    return (torch.cat(xs).contiguous(), torch.cat(ys).contiguous(), torch.cat(ps).contiguous(),
            torch.cat(coarse).contiguous())


def norm_stats(x, y):
    xm = x.reshape(-1, x.shape[-1]).mean(0)
    xs = x.reshape(-1, x.shape[-1]).std(0).clamp_min(1e-6)
    ys = y.reshape(-1, y.shape[-1]).std(0).clamp_min(1e-12)
    return xm.cpu().numpy(), xs.cpu().numpy(), ys.cpu().numpy()


def train(x, y, periodic, epochs=10, batch=256, lr=1e-3, seed=0, log=None, lr_final=None):
    """Trains a closure on device tensors; returns it and the per-epoch mean losses (each step's loss
    before its update).  The learning rate follows a cosine from lr down to lr_final (default lr / 20).
    Each epoch is one ql_closure_train_steps call: the mini-batches of a seeded permutation are gathered
    on the device, with no host round trip per step."""
    import torch
    xm, xsd, ysd = norm_stats(x, y)
    net = q.Closure(x.shape[2], y.shape[2], x.shape[1], batch, seed=seed, in_shift=xm, in_scale=xsd,
                    out_scale=ysd)
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    losses = []
    n = x.shape[0]
    per_epoch = n // batch
    lr_final = lr / 20.0 if lr_final is None else lr_final
    total = max(1, epochs * per_epoch)
    x, y = x.contiguous(), y.contiguous()
    per32 = periodic.to(torch.int32).contiguous()
    step_loss = torch.empty(per_epoch, dtype=torch.float32, device=x.device)
    for ep in range(epochs):
        perm = torch.randperm(n, device=x.device, generator=g)[:per_epoch * batch].to(torch.int32).contiguous()
        steps = np.arange(ep * per_epoch, (ep + 1) * per_epoch)
        rates = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * steps / total))
        net.train_steps(x, y, per32, perm, rates, step_loss)
        losses.append(float(step_loss.mean().item()) if per_epoch > 0 else 0.0)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return net, losses


def predict(net, x, periodic, batch):
    import torch
    out = torch.empty(x.shape[0], x.shape[1], 5, dtype=torch.float32, device=x.device)
    for s in range(0, x.shape[0], batch):
        e = min(s + batch, x.shape[0])
        net.forward(x[s:e].contiguous(), periodic[s:e].contiguous(), out[s:e])
    return out


def field_errors(pred_fields, ref_fields):
    """Max-norm and RMS error per field (device tensors [N][NC][5]) -> dict of floats."""
    d = (pred_fields - ref_fields).double()
    out = {}
    for i, f in enumerate(FIELDS):
        out[f] = {"linf": float(d[..., i].abs().max()), "l2": float(d[..., i].pow(2).mean().sqrt())}
    return out
