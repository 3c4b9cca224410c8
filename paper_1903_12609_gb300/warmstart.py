"""Learned warm start of the implicit step (include/fil_mlp.h): training data
from the plain solver, training of the per-filament network on the GPU with
the library's tensor-core kernels, and loading a trained network into a
solver context.

The network corrects the extrapolated initial guess X_0 of each 32-segment
filament (in the filament's own frame), for the extrapolation order it was
trained with (fil_set_extrapolation; stored with the weights, see
trained_order); inside fil_step the plain solve keeps
the last word (the start with the smaller residual is kept and a failed start
from the prediction is restarted from the extrapolation), so every step
converges to the same tolerance with or without it.

Train and evaluate (one GPU):
    python -m paper_1903_12609_gb300.warmstart --steps 4000 --out <file.npz>
    python -m paper_1903_12609_gb300.warmstart --trajectories 40 --steps 100 --out <file.npz>
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import fil
from .inputs import suspension

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_n32.npz")
SEG, NIN, NOUT = fil.MLP_SEG, fil.MLP_IN, fil.MLP_OUT


def make_context(n_fil, seed=0, stream=None, order=1, **over):
    """A solver context on the suspension workload (mixed precision,
    filament-RPY J0, extrapolation of the given order), initialised with
    straight filaments."""
    wl, base, t, mu, Fext, follower = suspension(n_fil, SEG, seed=seed)
    params = dict(a=wl.a, eta=wl.eta, dL=wl.dL, KB=wl.KB, KT=wl.KT, dt=wl.dt, tol=wl.tol,
                  max_iter=wl.max_iter, precision=fil.FIL_MIXED,
                  j0_model=fil.FIL_J0_FILAMENT_RPY)
    params.update(over)
    m = fil.Filaments(wl.seg_per_fil, stream=stream, **params)
    m.set_extrapolation(order)
    m.init_straight(base, t, mu, None)
    m.set_external(Fext, None, follower)
    return m, wl


def trained_order(path=DEFAULT_WEIGHTS):
    """The extrapolation order whose guess the stored network corrects (1 for
    weights saved before the order was recorded)."""
    z = np.load(path)
    return int(json.loads(str(z["meta"])).get("extrapolation_order", 1))


def record(torch, n_fil, n_steps, seed=0, skip=10, order=1):
    """Run the plain solver and keep, for every step after the first `skip`,
    the network inputs before the step and the targets after it (device
    tensors [n_steps * n_fil, 416] and [n_steps * n_fil, 192])."""
    m, _ = make_context(n_fil, seed, order=order)
    feat = torch.empty((n_steps, n_fil, NIN), dtype=torch.float32, device="cuda")
    targ = torch.empty((n_steps, n_fil, NOUT), dtype=torch.float32, device="cuda")
    iters = []
    for k in range(skip + n_steps):
        j = k - skip
        if j >= 0:
            m.warm_features(feat[j])
        iters.append(m.step())
        if j >= 0:
            m.warm_targets(targ[j])
    m.close()
    return feat.view(-1, NIN), targ.view(-1, NOUT), iters[skip:]


def residual_weights(wl):
    """How strongly an error in each output component moves the residual f
    (eqn RA-3d-system), per unit: Y_1 enters every position row with weight 1;
    u_n enters the rotation row n with weight 1 and, through the robot arm,
    the position rows of the segments beyond n with weight ~dL, i.e. ~dL (N - n)
    in total; Lambda enters only through the mobility, with weight
    ~(2/3) dt / (6 pi eta a)."""
    N = SEG
    w = np.empty(NOUT)
    w[0:3] = 1.0
    for n in range(N):
        w[3 + 3 * n:6 + 3 * n] = 1.0 + wl.dL * (N - n)
    w[3 + 3 * N:] = (2.0 / 3.0) * wl.dt / (6.0 * np.pi * wl.eta * wl.a)
    return w


def fit_norm(torch, feat, targ, weights=None, n_sample=200_000, seed=0):
    """Input normalisation: per-component mean and standard deviation from a
    random sample of rows (components that do not vary get std 1). Output
    normalisation: per-component mean; the scale is 1 / weight (times one
    global factor that gives the normalised targets unit mean square), so the
    loss weighs each component's error by its effect on the residual; with no
    weights, the per-component standard deviation."""
    rng = np.random.default_rng(seed)
    idx = torch.from_numpy(rng.choice(feat.shape[0], min(n_sample, feat.shape[0]),
                                      replace=False)).cuda()
    x = feat.index_select(0, idx).cpu().numpy().astype(np.float64)
    y = targ.index_select(0, idx).cpu().numpy().astype(np.float64)
    out = []
    for a, w in ((x, None), (y, weights)):
        mu, sd = a.mean(axis=0), a.std(axis=0)
        sd = np.where(sd > 1e-12 * max(1.0, np.abs(mu).max()), sd, 1.0)
        if w is not None:
            g = np.sqrt(np.mean((w * a.std(axis=0)) ** 2))
            sd = g / w
        out += [mu.astype(np.float32), sd.astype(np.float32)]
    return out            # in_mean, in_std, out_mean, out_std


def block_stats(targ_sample):
    """RMS of the targets per block (Y_1, u, Lambda) -- for the training log."""
    return {"Y1": float(np.sqrt(np.mean(targ_sample[:, :3] ** 2))),
            "u": float(np.sqrt(np.mean(targ_sample[:, 3:3 + 3 * SEG] ** 2))),
            "Lambda": float(np.sqrt(np.mean(targ_sample[:, 3 + 3 * SEG:] ** 2)))}


def init_params(seed=0):
    """He-normal hidden layers, a small output layer, zero biases."""
    rng = np.random.default_rng(seed)
    dims = [(NIN, 256), (256, 256), (256, 256), (256, NOUT)]
    p = []
    for l, (i, o) in enumerate(dims):
        s = np.sqrt(2.0 / i) * (0.1 if l == 3 else 1.0)
        p += [rng.standard_normal(i * o) * s, np.zeros(o)]
    return np.concatenate(p).astype(np.float32)


def train(torch, feat, targ, norm, epochs=4, batch=1024, lr=1e-3, seed=0, val_frac=0.05,
          log=None):
    """Adam with a cosine learning-rate decay over contiguous row blocks in a
    shuffled order; the last val_frac of the rows are held out. Returns
    (params, history)."""
    n = feat.shape[0]
    n_val = int(n * val_frac) // batch * batch
    n_tr = (n - n_val) // batch
    net = fil.fil_mlp_create(batch)
    fil.fil_mlp_set_norm(net, *norm)
    fil.fil_mlp_set_params(net, init_params(seed))
    rng = np.random.default_rng(seed)
    total = epochs * n_tr
    grad = torch.empty(fil.MLP_NPARAM, dtype=torch.float32, device="cuda")

    def val_loss():
        if n_val == 0:
            return float("nan")
        ls = []
        for b in range(n - n_val, n, batch):
            ls.append(fil.fil_mlp_gradients(net, feat[b:b + batch], targ[b:b + batch], batch, grad))
        return float(np.mean(ls))

    hist = {"val0": val_loss(), "train": [], "val": []}
    if log:
        log("validation loss of the initial network: %.4f" % hist["val0"])
    step = 0
    for ep in range(epochs):
        losses = []
        for blk in rng.permutation(n_tr):
            a = int(blk) * batch
            cur = lr * (0.05 + 0.95 * 0.5 * (1 + np.cos(np.pi * step / total)))
            losses.append(fil.fil_mlp_train_step(net, feat[a:a + batch], targ[a:a + batch], batch,
                                                 cur))
            step += 1
        hist["train"].append(float(np.mean(losses)))
        hist["val"].append(val_loss())
        if log:
            log("epoch %d: train %.4f  val %.4f" % (ep, hist["train"][-1], hist["val"][-1]))
    params = np.zeros(fil.MLP_NPARAM, dtype=np.float32)
    fil.fil_mlp_get_params(net, params)
    fil.fil_mlp_destroy(net)
    return params, hist


def save(path, params, norm, meta):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez_compressed(path, params=params, in_mean=norm[0], in_std=norm[1], out_mean=norm[2],
                        out_std=norm[3], meta=json.dumps(meta))


def load(path=DEFAULT_WEIGHTS, max_batch=1024, stream=None):
    """A fil_mlp handle with the stored parameters and normalisation (the
    caller destroys it with fil.fil_mlp_destroy)."""
    z = np.load(path)
    net = fil.fil_mlp_create(max_batch, stream)
    fil.fil_mlp_set_params(net, np.ascontiguousarray(z["params"], dtype=np.float32))
    fil.fil_mlp_set_norm(net, *(np.ascontiguousarray(z[k], dtype=np.float32)
                                for k in ("in_mean", "in_std", "out_mean", "out_std")))
    return net


def evaluate(torch, net, n_fil, n_steps, seed=1, warmup=5, order=1):
    """Per arm (the plain solve, and the network attached in each mode), all
    continuing from the same state after `warmup` plain steps: Broyden
    iterations per step, the mean of log10 ||f(X_0)||_inf (how close the start
    is), timesteps/s, and how often each candidate was taken."""
    m, wl = make_context(n_fil, seed, order=order)
    tol = wl.tol * wl.a
    for _ in range(warmup):
        m.step()
    S = n_fil * SEG
    st = [np.zeros((S, 3)), np.zeros((S, 4)), np.zeros((S, 3)), np.zeros((S, 3)),
          np.zeros((S - n_fil, 3))]
    m.get_state(*st)
    out = {}
    for name, use, mode in (("plain", False, 0),
                            ("best_of_two", True, fil.FIL_WARM_BEST_OF_TWO),
                            ("prediction_first", True, fil.FIL_WARM_PREDICTION_FIRST)):
        m.set_state(*st)
        fil.fil_warm_attach(m.ctx, net if use else None, mode)
        p0 = fil.fil_warm_stats(m.ctx)
        its, f0s = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_steps):
            f0s.append(m.broyden_begin())
            k, conv = 0, f0s[-1] <= tol
            while not conv:
                conv, _ = m.broyden_step()
                k += 1
            m.broyden_commit()
            its.append(k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        p1 = fil.fil_warm_stats(m.ctx)
        out[name] = {"iters_per_step": float(np.mean(its)),
                     "log10_f0": float(np.mean(np.log10(np.maximum(f0s, 1e-300)))),
                     "timesteps_per_s": n_steps / dt,
                     "from_prediction": p1[0] - p0[0], "from_extrapolation": p1[1] - p0[1]}
    fil.fil_warm_attach(m.ctx, None)
    m.close()
    return out


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-fil", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=4000,
                    help="recorded solver steps (per trajectory)")
    ap.add_argument("--trajectories", type=int, default=1,
                    help="independent suspensions recorded (seeds seed, seed + 1000, ...): many "
                         "short runs cover the early, nearly straight states a fresh suspension "
                         "starts from; one long run covers later, deformed states")
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--seed", type=int, default=100,
                    help="workload seed of the training trajectory (the bench uses seed 0)")
    ap.add_argument("--eval-steps", type=int, default=50)
    ap.add_argument("--extrapolation", type=int, default=1, choices=[1, 2, 3],
                    help="order of the extrapolated guess the network learns to correct")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    log = lambda s: print(s, flush=True)   # noqa: E731
    t0 = time.time()
    parts = [record(torch, args.n_fil, args.steps, seed=args.seed + 1000 * k,
                    order=args.extrapolation) for k in range(args.trajectories)]
    feat = torch.cat([f for f, _, _ in parts]) if len(parts) > 1 else parts[0][0]
    targ = torch.cat([t for _, t, _ in parts]) if len(parts) > 1 else parts[0][1]
    iters = [i for _, _, its in parts for i in its]
    del parts
    log("recorded %d x %d steps x %d filaments in %.1f s (plain: %.2f Broyden iterations/step)"
        % (args.trajectories, args.steps, args.n_fil, time.time() - t0, np.mean(iters)))
    wl = suspension(args.n_fil, SEG, seed=args.seed)[0]
    norm = fit_norm(torch, feat, targ, weights=residual_weights(wl), seed=args.seed)
    log("target RMS per block: %s" % json.dumps(block_stats(targ[:20000].cpu().numpy())))
    t1 = time.time()
    params, hist = train(torch, feat, targ, norm, epochs=args.epochs, batch=args.batch,
                         lr=args.lr, seed=args.seed, log=log)
    log("trained in %.1f s" % (time.time() - t1))
    del feat, targ
    meta = {"n_fil": args.n_fil, "steps": args.steps, "trajectories": args.trajectories,
            "epochs": args.epochs, "batch": args.batch, "lr": args.lr, "seed": args.seed,
            "extrapolation_order": args.extrapolation, "history": hist}
    save(args.out, params, norm, meta)
    net = load(args.out, max_batch=max(1024, args.n_fil))
    ev = evaluate(torch, net, args.n_fil, args.eval_steps, seed=args.seed + 1,
                  order=args.extrapolation)
    fil.fil_mlp_destroy(net)
    meta["evaluation"] = ev
    save(args.out, params, norm, meta)
    log(json.dumps(ev))


if __name__ == "__main__":
    main()
