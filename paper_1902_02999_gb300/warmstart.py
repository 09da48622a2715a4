"""Learned warm start for steady-state runs (include/maclab_ws.h).

A residual convolutional network proposes the starting state of a steady
run; the plain MacLABSWE iteration then converges from it and decides the
answer.  The network runs on a coarse grid (4 x 4 fine nodes per cell) and
is trained on steady states that the library's own batch solver produces.

Binding only: the network, its training step, the coarse encoding and the
fine decoding run in the library's kernels (warmstart.cu); torch provides
device memory.

    python -m paper_1902_02999_gb300.warmstart --train 1024 --test 32

trains on seeded dish lakes and reports steps and wall time to residual
1e-8 from rest and from the proposal.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import time

import numpy as np

from . import Batch, MaclabError, _abi, lib

IO = 16
CELL = 4
# dilations of the residual blocks: receptive field wider than the 64 x 64 grid
DEFAULT_DILATIONS = (1, 2, 4, 8, 16, 32, 1, 2, 4, 8, 16, 1)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class WarmStartNet:
    """One network handle (maclab_ws_t) with its own weights and buffers."""

    def __init__(self, res: int = 64, channels: int = 128, dilations=DEFAULT_DILATIONS, max_batch: int = 32,
                 seed: int = 0, stream=None, tensor_path: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the warm start needs a CUDA GPU; no CPU fallback exists")
        self._lib = lib()
        self.res, self.channels, self.dilations = res, channels, tuple(dilations)
        self.max_batch = max_batch
        cfg = _abi.WSConfig()
        cfg.res, cfg.channels, cfg.blocks, cfg.max_batch, cfg.seed = res, channels, len(dilations), max_batch, seed
        # the 128 -> 128 convolutions on 0: tcgen05 fed by TMA, 1: tcgen05 fed
        # by cp.async, 2: mma.sync
        cfg.tensor_path = tensor_path
        for k, d in enumerate(dilations):
            cfg.dilation[k] = int(d)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.maclab_ws_create(ctypes.byref(cfg), ctypes.c_void_p(int(stream.cuda_stream)), ctypes.byref(h))
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_last_error(None).decode())
        self._h = h
        n = ctypes.c_int64()
        self._check(self._lib.maclab_ws_param_count(self._h, ctypes.byref(n)))
        self.nparam = n.value

    def _check(self, rc):
        if rc != 0:
            raise MaclabError(rc, self._lib.maclab_last_error(None).decode())

    # ---- parameters
    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        self._check(self._lib.maclab_ws_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                   self.nparam))
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        assert t.size == self.nparam
        self._check(self._lib.maclab_ws_set_params(self._h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                   self.nparam))

    # ---- network
    def forward(self, x):
        import torch
        y = torch.empty_like(x)
        self._check(self._lib.maclab_ws_forward(self._h, x.shape[0], _ptr(x), _ptr(y)))
        return y

    def gradients(self, x, t, w, out_ch: int = 3):
        g = np.empty(self.nparam, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.maclab_ws_gradients(self._h, x.shape[0], out_ch, _ptr(x), _ptr(t), _ptr(w),
                                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.nparam,
                                                  ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, x, t, w, lr: float, out_ch: int = 3, want_loss: bool = True):
        loss = ctypes.c_double()
        self._check(self._lib.maclab_ws_train_step(self._h, x.shape[0], out_ch, _ptr(x), _ptr(t), _ptr(w),
                                                   float(lr), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    # ---- single-layer checks
    def keep_gradients(self, on: bool = True) -> None:
        """Keep the loss gradient with respect to every H_l after the next
        gradients or train step (for inspect(1, l, ...))."""
        self._check(self._lib.maclab_ws_keep_gradients(self._h, int(bool(on))))

    def inspect(self, what: int, index: int, batch: int):
        """A stored tensor as float on the device: 0 H_{index+1}, 1 its loss
        gradient (keep_gradients on), 2 the loss gradient of Y, 3 Y."""
        import torch
        ch = self.channels if what in (0, 1) else 16
        out = torch.empty((batch, self.res, self.res, ch), dtype=torch.float32, device="cuda")
        self._check(self._lib.maclab_ws_inspect(self._h, what, index, batch, _ptr(out), out.numel()))
        return out

    # ---- fine <-> coarse
    def encode(self, D, mask, case, scale, state=None):
        """Coarse input x [R][R][16] (and, with state = (eta, u, v, pitch)
        device pointers, targets t [R][R][16] and weights w [R][R])."""
        import torch
        R = self.res
        dev = D.device
        x = torch.empty((R, R, IO), dtype=torch.float32, device=dev)
        t = w = None
        sc = (ctypes.c_double * 4)(*scale)
        if state is not None:
            t = torch.empty((R, R, IO), dtype=torch.float32, device=dev)
            w = torch.empty((R, R), dtype=torch.float32, device=dev)
            eta, u, v, pitch = state
        else:
            eta = u = v = None
            pitch = 0
        self._check(self._lib.maclab_ws_encode(
            self._h, R * CELL, _ptr(D), _ptr(mask), float(case.wind_u), float(case.wind_v), float(case.cb),
            float(case.dx), ctypes.c_void_p(eta), ctypes.c_void_p(u), ctypes.c_void_p(v), int(pitch), sc,
            _ptr(x), _ptr(t) if t is not None else None, _ptr(w) if w is not None else None))
        return x, t, w

    def decode(self, y, D, mask, scale, mass_eta=float("nan")):
        """Fine proposal (h, u, v) as float64 device tensors [n][n]; with a
        finite mass_eta, eta sums to it over the non-solid nodes."""
        import torch
        n = self.res * CELL
        h, u, v = (torch.empty((n, n), dtype=torch.float64, device=D.device) for _ in range(3))
        sc = (ctypes.c_double * 4)(*scale)
        self._check(self._lib.maclab_ws_decode(self._h, n, _ptr(y), _ptr(D), _ptr(mask), sc, float(mass_eta),
                                               _ptr(h), _ptr(u), _ptr(v)))
        return h, u, v

    def close(self):
        if getattr(self, "_h", None):
            self._lib.maclab_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
def lake_fields(case, device):
    """Still-water depth D = h_ref - z_b (float32) and the mask on the device."""
    import torch
    D = torch.tensor(np.asarray(case.h_ref - case.zb, dtype=np.float32), device=device)
    M = torch.tensor(np.asarray(case.mask, dtype=np.uint8), device=device)
    return D, M


def steady_batch(cases, tol=1e-8, max_steps=200000, check_every=1000):
    """Plain iteration of every case to residual tol in one batch; returns
    the batch (kept alive for its device states) and steps / seconds."""
    b = Batch(cases, precision="f32")
    steps, r, sec = b.run_to_steady(tol=tol, max_steps=max_steps, check_every=check_every)
    return b, steps, r, sec


def make_dataset(net, cases, tol=1e-7, max_steps=120000, chunk=1024, scale=None):
    """Steady states of `cases` (plain iteration, FP32) encoded for training:
    X, T [N][R][R][16], W [N][R][R] on the device, the scales used and the
    per-case steps.  Targets are taken at residual `tol` (or max_steps)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    R = net.res
    N = len(cases)
    X = torch.empty((N, R, R, IO), dtype=torch.float32, device=dev)
    T = torch.empty_like(X)
    W = torch.empty((N, R, R), dtype=torch.float32, device=dev)
    raw = scale is None
    sc = (1.0, 1.0, 1.0, 1.0) if raw else scale
    all_steps = np.zeros(N, dtype=np.int64)
    for c0 in range(0, N, chunk):
        part = cases[c0:c0 + chunk]
        b, steps, _, _ = steady_batch(part, tol=tol, max_steps=max_steps)
        all_steps[c0:c0 + len(part)] = steps
        for k, case in enumerate(part):
            D, M = lake_fields(case, dev)
            x, t, w = net.encode(D, M, case, sc, state=b.device_state(k))
            X[c0 + k], T[c0 + k], W[c0 + k] = x, t, w
        torch.cuda.synchronize()
        b.close()
    if raw:
        # divisors that make the target channels O(1) and the depth channel O(1)
        live = W > 0
        s_eta = float(T[..., 0][live].std().item()) or 1.0
        s_u = float(torch.sqrt((T[..., 1][live] ** 2 + T[..., 2][live] ** 2).mean()).item()) or 1.0
        dmax = float(max(np.max(c.h_ref - c.zb) for c in cases))
        sc = (dmax, s_eta, s_u, s_u)
        X[..., 1] /= sc[0]
        T[..., 0] /= sc[1]
        T[..., 1] /= sc[2]
        T[..., 2] /= sc[3]
    return X, T, W, sc, all_steps


def train(net, X, T, W, epochs=30, batch=16, lr=1e-3, seed=0, log=None):
    """Adam over shuffled mini-batches with a cosine learning rate; the
    sample weights are normalised to sum to one per batch."""
    import torch
    N = X.shape[0]
    rng = np.random.default_rng(seed)
    steps_total = epochs * max(1, N // batch)
    k = 0
    losses = []
    for ep in range(epochs):
        order = rng.permutation(N)
        ep_loss = 0.0
        for i in range(0, N - batch + 1, batch):
            idx = torch.as_tensor(order[i:i + batch], device=X.device)
            xb, tb, wb = X[idx].contiguous(), T[idx].contiguous(), W[idx]
            wb = (wb / wb.sum()).contiguous()
            lr_k = 0.5 * lr * (1.0 + math.cos(math.pi * k / steps_total))
            ep_loss += net.train_step(xb, tb, wb, lr_k)
            k += 1
        losses.append(ep_loss / max(1, N // batch))
        if log:
            log("epoch %d loss %.4e" % (ep, losses[-1]))
    return losses


def closed_basin(case) -> bool:
    """No Dirichlet node: the iteration conserves the volume exactly."""
    return not np.isin(np.asarray(case.mask), (3, 4, 5)).any()


def propose(net, case, scale):
    """Warm-start state (h, u, v) of one case as host float64 arrays.  In a
    closed basin the proposal keeps the still-water volume (sum eta = 0)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    D, M = lake_fields(case, dev)
    x, _, _ = net.encode(D, M, case, scale)
    y = net.forward(x.unsqueeze(0))[0].contiguous()
    h, u, v = net.decode(y, D, M, scale, 0.0 if closed_basin(case) else float("nan"))
    return h.cpu().numpy(), u.cpu().numpy(), v.cpu().numpy()


def _rel_err(case, state, ref_state):
    """Max relative errors (eta, velocity) of a state against a reference, over
    non-solid nodes: eta by max|eta_ref|, u and v by the largest reference speed."""
    live = case.mask != 0
    D = case.h_ref - case.zb
    eta, eta_r = state[0] - D, ref_state[0] - D
    e_eta = np.abs(eta - eta_r)[live].max() / max(np.abs(eta_r)[live].max(), 1e-30)
    sp = np.hypot(ref_state[1], ref_state[2])[live].max()
    e_u = max(np.abs(state[1] - ref_state[1])[live].max(), np.abs(state[2] - ref_state[2])[live].max()) / max(sp, 1e-30)
    return e_eta, e_u


def _timed_steps(batch, k):
    """Advance a batch k steps; device time (ms) from CUDA events."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    batch.step(k)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def _run_to_accuracy(batch, cases, refs, targets, max_steps, check_every):
    """Step until every instance is within its target errors of its
    reference state (checked every check_every steps on the host); returns
    the steps per instance (-1: not reached) and the device time spent."""
    n = len(cases)
    done = np.full(n, -1, dtype=np.int64)
    act = np.ones(n, dtype=bool)
    steps, ms = 0, 0.0
    while act.any() and steps < max_steps:
        ms += _timed_steps(batch, check_every)
        steps += check_every
        for i in np.where(act)[0]:
            e = _rel_err(cases[i], batch.get_state(i), refs[i])
            if e[0] <= targets[i][0] and e[1] <= targets[i][1]:
                done[i] = steps
                act[i] = False
        batch.set_active(act.astype(np.uint8))
    return done, ms


def compare(net, cases, scale, tol=1e-8, max_steps=400000, check_every=500, ref_tol=1e-11):
    """The plain iteration from rest and from the network's proposal, both
    FP32 batches of the same cases on the same GPU.

    Errors are measured against an FP64 run of the plain iteration to
    residual ref_tol (the FP64 path equals the FP64 oracle to 1e-12).
      plain:  steps and wall time to residual tol from rest, and the error
              reached there;
      warm_residual: steps to residual tol from the proposal and the error
              reached there (the residual can fall below tol while a slow
              large-scale mode still carries more error than the plain run
              has when it stops);
      warm_matched: steps from the proposal until the state is as close to
              the FP64 steady state as the plain run's final state (eta and
              velocity), and the device time of those steps plus the time
              to make the proposal."""
    import torch
    ref = Batch(cases, precision="f64")
    sr, _, _ = ref.run_to_steady(tol=ref_tol, max_steps=4 * max_steps, check_every=check_every)
    states_ref = [ref.get_state(i) for i in range(len(cases))]
    ref.close()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = Batch(cases, precision="f32")
    sp, _, secp = plain.run_to_steady(tol=tol, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall_plain = time.perf_counter() - t0
    plain_err = np.array([_rel_err(c, plain.get_state(i), r) for i, (c, r) in enumerate(zip(cases, states_ref))])
    # device time per batch step of these cases (every instance active)
    plain.set_active(np.ones(len(cases), dtype=np.uint8))
    ms_per_step = _timed_steps(plain, 200) / 200
    plain.close()

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    proposals = [propose(net, c, scale) for c in cases]
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    prop_err = np.array([_rel_err(c, p, r) for c, p, r in zip(cases, proposals, states_ref)])

    warm = Batch(cases, precision="f32")
    for i, p in enumerate(proposals):
        warm.set_state(i, *p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sw, _, secw = warm.run_to_steady(tol=tol, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall_warm_residual = time.perf_counter() - t0 + t_prop
    warm_err = np.array([_rel_err(c, warm.get_state(i), r) for i, (c, r) in enumerate(zip(cases, states_ref))])
    warm.close()

    # the same residual rule ten times tighter: still a rule a user can
    # apply without a reference solution
    warm = Batch(cases, precision="f32")
    for i, p in enumerate(proposals):
        warm.set_state(i, *p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st10, _, _ = warm.run_to_steady(tol=tol / 10, max_steps=max_steps, check_every=check_every)
    torch.cuda.synchronize()
    wall_warm_tight = time.perf_counter() - t0 + t_prop
    tight_err = np.array([_rel_err(c, warm.get_state(i), r) for i, (c, r) in enumerate(zip(cases, states_ref))])
    warm.close()

    warm = Batch(cases, precision="f32")
    for i, p in enumerate(proposals):
        warm.set_state(i, *p)
    sm, ms_matched = _run_to_accuracy(warm, cases, states_ref, plain_err, max_steps, check_every)
    warm.close()
    return {"plain_steps": sp, "plain_seconds": secp, "wall_plain": wall_plain, "plain_error": plain_err,
            "ref_steps": sr, "proposal_error": prop_err, "proposal_seconds": t_prop,
            "warm_steps": sw, "warm_seconds": secw, "wall_warm_residual": wall_warm_residual,
            "warm_error": warm_err, "warm_tight_steps": st10, "wall_warm_tight": wall_warm_tight,
            "warm_tight_error": tight_err, "tol": tol,
            "matched_steps": sm, "wall_warm_matched": ms_matched / 1e3 + t_prop,
            "ms_per_step": ms_per_step}


def _headline(res):
    """The warm start at a stopping rule a user can apply: the residual
    tolerance itself if the warm runs' largest errors (eta, velocity
    against the FP64 steady state) are within the plain runs', else the
    tolerance ten times tighter if they are; wall times on the same host
    clock (from the call's start, syncs included), the proposal included."""
    plain = res["plain_error"].max(axis=0)
    for key, err, wall, steps, tol in (
            ("residual_only", res["warm_error"], res["wall_warm_residual"], res["warm_steps"], res["tol"]),
            ("residual_tight", res["warm_tight_error"], res["wall_warm_tight"], res["warm_tight_steps"],
             res["tol"] / 10)):
        if (err.max(axis=0) <= plain).all() and (steps > 0).all():
            return {"rule": "warm run to residual %g (plain run to %g)" % (tol, res["tol"]), "from": key,
                    "wall_warm_s": wall, "wall_plain_s": res["wall_plain"],
                    "wall_ratio": res["wall_plain"] / wall,
                    "error_max_warm": err.max(axis=0).tolist(), "error_max_plain": plain.tolist(),
                    "clock": "host wall clock around each batch run (residual syncs included)"}
    return {"rule": None, "note": "no residual rule tried reaches the plain runs' accuracy"}


def summary(res):
    """JSON-friendly medians / maxima of a compare() result."""
    med = lambda x: float(np.median(x)) if len(x) else None
    okp = res["plain_steps"] > 0
    okm = okp & (res["matched_steps"] > 0)
    okw = okp & (res["warm_steps"] > 0)
    return {"cases": int(len(okp)), "plain_converged": int(okp.sum()),
            "plain_steps_median": med(res["plain_steps"][okp]),
            "wall_plain_s": res["wall_plain"],
            "plain_error_max": res["plain_error"].max(axis=0).tolist(),
            "matched": {"reached": int(okm.sum()), "steps_median": med(res["matched_steps"][okm]),
                        "steps_ratio_median": med(res["plain_steps"][okm] / res["matched_steps"][okm]),
                        "wall_s": res["wall_warm_matched"]},
            "residual_only": {"converged": int(okw.sum()), "steps_median": med(res["warm_steps"][okw]),
                              "wall_s": res["wall_warm_residual"],
                              "error_max": res["warm_error"].max(axis=0).tolist()},
            "residual_tight": {"tol": res["tol"] / 10, "converged": int((res["warm_tight_steps"] > 0).sum()),
                               "steps_median": med(res["warm_tight_steps"][res["warm_tight_steps"] > 0]),
                               "wall_s": res["wall_warm_tight"],
                               "error_max": res["warm_tight_error"].max(axis=0).tolist()},
            "headline": _headline(res),
            "proposal_s": res["proposal_seconds"], "ms_per_batch_step": res["ms_per_step"],
            "proposal_error_median": np.median(res["proposal_error"], axis=0).tolist()}


def time_kernels(batch: int = 16, reps: int = 50, paths=(0, 2)) -> dict:
    """Forward and training-step times of the default network on random
    inputs, per convolution path (0: tcgen05 fed by TMA, 1: tcgen05 fed by
    cp.async, 2: mma.sync), with CUDA events on the current stream.  The
    FLOP rates count 2 per multiply-add of the convolutions (a training
    step: forward, input gradient and weight gradient, three times the
    forward)."""
    import torch
    out = {}
    for path in paths:
        net = WarmStartNet(max_batch=batch, tensor_path=path)
        g = torch.Generator(device="cuda").manual_seed(0)
        R = net.res
        X = torch.randn(batch, R, R, IO, device="cuda", generator=g)
        T = torch.randn(batch, R, R, IO, device="cuda", generator=g)
        Wt = torch.full((batch, R, R), 1.0 / (batch * R * R), device="cuda")
        for _ in range(5):
            net.train_step(X, T, Wt, 1e-4, want_loss=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.train_step(X, T, Wt, 1e-4, want_loss=False)
        e1.record()
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1) / reps
        e0.record()
        for _ in range(reps):
            net.forward(X)
        e1.record()
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1) / reps
        C, L = net.channels, len(net.dilations)
        flop = 2.0 * batch * R * R * 9 * (IO * C + L * C * C + C * IO)
        out["path%d" % path] = {"forward_ms": fwd_ms, "train_step_ms": train_ms,
                                "forward_tflops": flop / fwd_ms / 1e9, "train_tflops": 3 * flop / train_ms / 1e9}
        net.close()
    return out


def main():
    import torch
    import inputs
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--test", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--target-tol", type=float, default=1e-7)
    ap.add_argument("--time-kernels", action="store_true",
                    help="only time the network's forward pass and training step per convolution path")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    if args.time_kernels:
        print(json.dumps({"batch": args.batch, **time_kernels(args.batch)}))
        return
    net = WarmStartNet(max_batch=args.batch)
    t0 = time.perf_counter()
    train_cases = [inputs.dish_lake(256, seed=1000 + k) for k in range(args.train)]
    X, T, W, scale, steps = make_dataset(net, train_cases, tol=args.target_tol)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = train(net, X, T, W, epochs=args.epochs, batch=args.batch, lr=args.lr, log=print)
    t_train = time.perf_counter() - t0
    test_cases = [inputs.dish_lake(256, seed=k) for k in range(args.test)]
    res = compare(net, test_cases, scale)
    out = {"train": args.train, "epochs": args.epochs, "params": net.nparam, "data_s": t_data,
           "train_s": t_train, "loss_first": losses[0], "loss_last": losses[-1], "scale": list(scale),
           "data_steps_median": float(np.median(steps[steps > 0])) if (steps > 0).any() else None}
    out.update(summary(res))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
