"""The shape of the paper's preconditioner / Laplacian / step-size comparison
(Sec. 5.1.2: Tables 3, 4 and 5, and the convergence-rate figure) on a
synthetic image with ground truth.

The paper segments a photograph ('stone') with eps = 100, c = 11, eta = 100,
a 25 x 25 search window and 4 preconditioned sweeps per outer step, and
counts the outer steps (and seconds) a configuration needs.  Its stopping
rule is a stable DICE score against the ground truth: the score varies by at
most 1e-5 over 10 consecutive steps.  Here the image is a seeded ellipse
image with noise (ground truth known) and its graph the window k-NN patch
graph built on the GPU (pdca_image_graph, 25 x 25 window).

    python -m paper_2303_14495_gb300.study [--size 256] [--json out.json]

Each configuration runs outer steps of 4 sweeps (pdca_step) until the DICE
score is stable or max_outer; the time is the device time of those steps
(CUDA events; the DICE evaluation in between is not timed).  The rate
experiment runs the reference configuration (normalized L_s, perturbed
Jacobi, infinite step size) for many steps, takes the last iterate as u*,
and reports ||u^t - u*|| / ||u*|| at t = 1, 2, 4, ... with the log-log
slope.
"""

from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import binding as B

EPS, C, ETA, INNER = 100.0, 11.0, 100.0, 4


def dice(lab: np.ndarray, gt: np.ndarray) -> float:
    a = lab == 1
    b = gt == 1
    s = a.sum() + b.sum()
    return 1.0 if s == 0 else 2.0 * float(np.logical_and(a, b).sum()) / float(s)


def build_case(size: int = 256, seed: int = 2303, label_frac: float = 0.02, window_radius: int = 12,
               patch_radius: int = 1, k: int = 10, sigma: float = 0.5, noise: float = 0.15):
    """(row_ptr, col, w) on the device, ground truth, fidelity mask and labels."""
    import torch
    from gen.workloads import ellipse_image, sample_labels
    rng = np.random.default_rng(seed)
    img, gt = ellipse_image(size, 6, noise, rng)
    rp, col, w = B.image_graph(torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda(), patch_radius,
                               window_radius, k, sigma)
    gt = gt.ravel().astype(np.int32)
    mask, lab = sample_labels(gt, label_frac, 2, rng)
    return (rp, col, w), gt, mask, lab


def run_config(graph, gt, mask, lab, laplacian: int, precond: int, step_k: float, max_outer: int = 3000,
               window: int = 10, tol: float = 1e-5):
    """Outer steps until the DICE score of the last `window` steps varies by
    at most tol; returns (steps or None, device ms, final DICE)."""
    import torch
    rp, col, w = graph
    prm = B.make_params(eps=EPS, c=C, eta=ETA, precond=precond, damping=0.5, laplacian=laplacian, step_k=step_k)
    g = B.Problem(rp, col, w, 1, mask, lab, prm)
    stream = torch.cuda.current_stream()
    ms = 0.0
    d = 0.0
    hist = []
    for t in range(1, max_outer + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.step(INNER)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
        d = dice(g.labels(), gt)
        hist.append(d)
        if t >= window and max(hist[-window:]) - min(hist[-window:]) <= tol:
            g.close()
            return t, ms, d
    g.close()
    return None, ms, d


def plateau(graph, gt, mask, lab, steps: int = 2000):
    """DICE and iterate of the reference configuration after many steps."""
    rp, col, w = graph
    prm = B.make_params(eps=EPS, c=C, eta=ETA, precond=B.PDCA_JACOBI_PERTURBED)
    g = B.Problem(rp, col, w, 1, mask, lab, prm)
    g.solve(steps, INNER)
    u = g.get_u().astype(np.float64)
    d = dice(g.labels(), gt)
    g.close()
    return d, u


def rate(graph, gt, mask, lab, u_star, steps: int = 1024):
    rp, col, w = graph
    prm = B.make_params(eps=EPS, c=C, eta=ETA, precond=B.PDCA_JACOBI_PERTURBED)
    g = B.Problem(rp, col, w, 1, mask, lab, prm)
    out, t, nxt = [], 0, 1
    while t < steps:
        g.step(INNER)
        t += 1
        if t == nxt:
            out.append((t, float(np.linalg.norm(g.get_u() - u_star) / np.linalg.norm(u_star))))
            nxt *= 2
    g.close()
    ts = np.log([a for a, _ in out if _ > 0])
    es = np.log([e for _, e in out if e > 0])
    slope = float(np.polyfit(ts, es, 1)[0]) if len(ts) >= 2 else float("nan")
    return out, slope


def study(size: int = 256, max_outer: int = 3000, verbose: bool = True, noise: float = 0.15):
    graph, gt, mask, lab = build_case(size, noise=noise)
    d_star, u_star = plateau(graph, gt, mask, lab)
    if verbose:
        print(f"image {size}x{size}: DICE of u* (reference, 2000 steps) {d_star:.4f}", file=sys.stderr)
    Jp, Jd, R = B.PDCA_JACOBI_PERTURBED, B.PDCA_JACOBI_DAMPED, B.PDCA_RICHARDSON
    rows = []

    def one(table, name, lap, pc, k):
        steps, ms, d = run_config(graph, gt, mask, lab, lap, pc, k, max_outer)
        rows.append(dict(table=table, config=name, laplacian="L_s" if lap == 0 else "L",
                         precond={Jp: "perturbed", Jd: "damped", R: "Richardson"}[pc],
                         step="inf" if k == 0 else k, steps=steps, ms=round(ms, 2), dice=round(d, 4)))
        if verbose:
            print(f"  {table} {name:28s} steps {steps} ms {ms:.1f} DICE {d:.4f}", file=sys.stderr)

    one("3", "perturbed, L_s", 0, Jp, 0.0)
    one("3", "perturbed, L", 1, Jp, 0.0)
    for name, pc in [("perturbed", Jp), ("damped", Jd), ("Richardson", R)]:
        one("4", f"{name}, L_s", 0, pc, 0.0)
    for pc, name in [(Jp, "perturbed"), (R, "Richardson")]:
        for k in (0.01, 0.05, 0.1, 1.0, 5.0, 0.0):
            one("5", f"{name}, L_s, k={'inf' if k == 0 else k}", 0, pc, k)
    curve, slope = rate(graph, gt, mask, lab, u_star)
    return dict(size=size, eps=EPS, c=C, eta=ETA, inner=INNER, stop="DICE within 1e-5 over 10 steps",
                dice_u_star=d_star, runs=rows, rate=dict(points=curve, loglog_slope=slope))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--max-outer", type=int, default=3000)
    ap.add_argument("--noise", type=float, default=0.15)
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    res = study(a.size, a.max_outer, noise=a.noise)
    s = json.dumps(res, indent=1)
    if a.json:
        with open(a.json, "w") as f:
            f.write(s)
    print(s)


if __name__ == "__main__":
    main()
