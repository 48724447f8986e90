"""Offline sweep of the BF16 tensor-core passes' launch shapes.

For each tuning key (pass, row bucket, MMA width, n class; see tt_tune_set
in include/tt_rbki.h) one representative unfolding is timed under every
candidate entry: ring depth, CTAs per SM, and the Gram's stage width or the
tall projection's chunk height.  A time is that of the whole pass (every
kernel of the call: operand preparation, the pass, the sum of its per-CTA
partials, whose count follows the grid): `--reps` calls captured in one
CUDA graph, replayed twice untimed and then timed by CUDA events around
three replays, on seeded Gaussian BF16 data.  An
entry is written only where the fastest candidate beats the built-in rules
by more than `--gain` (3%); every candidate's output is first checked
against the built-in shape's output (same pass, so the difference is the
order of FP32 partial sums).

    python -m paper_2308_01480_gb300.autotune [--out FILE] [--reps 10]

The table the library loads is paper_2308_01480_gb300/tune_table.txt
(`_native.TUNE_TABLE`).  Needs a GPU.
"""
import argparse
import datetime
import itertools
import sys

import torch

import paper_2308_01480_gb300 as tt
from paper_2308_01480_gb300 import _native as N

NAME = {N.TT_PASS_SKETCH: "sketch", N.TT_PASS_GRAMAPPLY: "gram_apply", N.TT_PASS_PROJECT: "project",
        N.TT_PASS_GRAM: "gram"}

# (pass, m, n, b): the unfoldings of the 40^5 and 256x256x64x32 workloads'
# tensor-core passes, and one large case per further row bucket
SHAPES = [
    (N.TT_PASS_GRAM, 40, 2560000, 0),
    (N.TT_PASS_GRAM, 16, 8388608, 0),
    (N.TT_PASS_GRAM, 64, 2097152, 0),
    (N.TT_PASS_GRAM, 128, 1048576, 0),
    (N.TT_PASS_GRAM, 40, 8192, 0),
    (N.TT_PASS_PROJECT, 40, 2560000, 20),
    (N.TT_PASS_PROJECT, 800, 64000, 20),
    (N.TT_PASS_PROJECT, 800, 1600, 20),
    (N.TT_PASS_PROJECT, 256, 524288, 30),
    (N.TT_PASS_PROJECT, 128, 1048576, 30),
    (N.TT_PASS_SKETCH, 800, 64000, 30),
    (N.TT_PASS_SKETCH, 800, 1600, 30),
    (N.TT_PASS_SKETCH, 256, 524288, 40),
    (N.TT_PASS_SKETCH, 40, 2560000, 30),
    (N.TT_PASS_GRAMAPPLY, 256, 524288, 40),
    (N.TT_PASS_GRAMAPPLY, 128, 1048576, 32),
    (N.TT_PASS_GRAMAPPLY, 800, 64000, 30),
]


def candidates(op, m):
    stages = (2, 3, 4, 6, 8)
    out = []
    for st, per in itertools.product(stages, (1, 2)):
        if op == N.TT_PASS_GRAM:
            out += [(st, per, kb, 0) for kb in (1, 2, 4, 8)]
        elif op == N.TT_PASS_PROJECT and m > 128:
            out += [(st, per, 0, cr) for cr in (64, 128)]
        else:
            out.append((st, per, 0, 0))
    return out


def _inputs(op, m, n, b, g):
    C = torch.randn(m, n, device="cuda", generator=g).to(torch.bfloat16)
    if op == N.TT_PASS_SKETCH:
        X = torch.randn(n, b, device="cuda", generator=g)
    elif op == N.TT_PASS_GRAM:
        X = None
    else:
        X = torch.randn(m, b, device="cuda", generator=g)
    return C, X


def _time(op, C, X, out, ws, reps):
    """Microseconds per call of the whole pass, from a graph of `reps` calls."""
    kw = dict(y_dtype=torch.bfloat16) if op == N.TT_PASS_PROJECT else {}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        tt.tt_pass(op, C, x=X, out=out, workspace=ws, stream=s, **kw)     # shapes and maps built once
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for _ in range(reps):
                tt.tt_pass(op, C, x=X, out=out, workspace=ws, stream=s, **kw)
        for _ in range(2):
            g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(3):
            g.replay()
        e1.record(s)
        s.synchronize()
    del g
    return 1000.0 * e0.elapsed_time(e1) / (3 * reps)


def _bound(op, C, X):
    """max of the |.|-product bound of the pass (the scale of its rounding)."""
    a = C.float().abs()
    if op == N.TT_PASS_GRAM:
        return (a @ a.T).max().item()
    x = X.abs()
    if op == N.TT_PASS_SKETCH:
        return (a @ x).max().item()
    if op == N.TT_PASS_GRAMAPPLY:
        return (a @ (a.T @ x)).max().item()
    return (x.T @ a).max().item()


def _close(op, y, ref, bound):
    """The same pass under another launch shape: equal up to the order of
    FP32 partial sums, with the tolerances of the pass tests (relative to the
    |.|-product bound; a BF16 projection output also up to one rounding)."""
    d = (y.float() - ref.float()).abs().max().item()
    if op == N.TT_PASS_PROJECT:
        return d <= 2 ** -7 * ref.float().abs().max().item() + 1e-5 * bound
    return d <= (2e-4 if op == N.TT_PASS_GRAMAPPLY else 1e-5) * bound


def sweep(reps=10, gain=0.03, log=sys.stdout):
    tt._native.lib()
    tt.tune_clear()
    g = torch.Generator(device="cuda").manual_seed(20230803)
    lines = []
    for op, m, n, b in SHAPES:
        key = tt.tune_key(op, m, n, b)
        C, X = _inputs(op, m, n, b, g)
        kw = dict(y_dtype=torch.bfloat16) if op == N.TT_PASS_PROJECT else {}
        tt.tune_clear()
        ref = tt.tt_pass(op, C, x=X, **kw).clone()
        bound = _bound(op, C, X)
        out = torch.empty_like(ref)
        ws = torch.empty(tt.pass_workspace_size(op, m, n, b, N.TT_BF16), dtype=torch.uint8, device="cuda")
        base = _time(op, C, X, out, ws, reps)
        best, best_us = None, base
        for cand in candidates(op, m):
            tt.tune_clear()
            tt.tune_set(key, *cand)
            y = tt.tt_pass(op, C, x=X, out=out, workspace=ws, **kw)
            if not _close(op, y, ref, bound):
                raise RuntimeError(f"{NAME[op]} {m}x{n} b={b} entry {cand}: output differs from the built-in shape")
            us = _time(op, C, X, out, ws, reps)
            if us < best_us:
                best, best_us = cand, us
        tt.tune_clear()
        gb = (m * n * 2) / (best_us * 1e3)
        print(f"{NAME[op]:10s} {m:5d} x {n:8d} b={b:3d} key={key}: built-in {base:8.1f} us, best {best_us:8.1f} us "
              f"{best}", file=log, flush=True)
        what = f"{NAME[op]} {m} x {n}, b = {b}: built-in {base:.1f} us, tuned {best_us:.1f} us ({gb:.0f} GB/s of C)"
        if best is not None and best_us < (1.0 - gain) * base:
            lines.append((key, best, what))
        else:
            lines.append((key, None, what + "; built-in kept"))
        del C, X, ref, out, ws
        torch.cuda.empty_cache()
    return lines


def write_table(lines, path):
    dev = torch.cuda.get_device_name(0)
    with open(path, "w") as f:
        f.write("# Launch shapes of the BF16 tensor-core passes (tt_tune_load format:\n")
        f.write("# op rows npad nclass stages per_sm kb chunk_rows), written by\n")
        f.write("# `python -m paper_2308_01480_gb300.autotune` on " + dev + ", "
                + datetime.date.today().isoformat() + ".\n")
        f.write("# Per-launch CUDA-event times of one representative unfolding per key.\n")
        for key, best, what in lines:
            if best is None:
                f.write(f"# {' '.join(map(str, key))}: {what}\n")
            else:
                f.write(" ".join(map(str, key + best)) + f"   # {what}\n")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out", default=N.TUNE_TABLE)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--gain", type=float, default=0.03)
    a = ap.parse_args(argv)
    lines = sweep(a.reps, a.gain)
    write_table(lines, a.out)
    tt.tune_load(a.out)
    print(f"wrote {a.out} ({tt.tune_entries()} entries)")


if __name__ == "__main__":
    main()
