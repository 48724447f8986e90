"""The paper's synthetic accuracy study (Sec. 4.1, 4.2) on the GPU: time,
relative error and PSNR of TT-rBKI (Alg. 3; also with the accurate_rr
Rayleigh-Ritz, tt_rbki_acc), TT-rSI (Alg. 4), TT-rSVD (Alg. 2) and TT-SVD
(Alg. 1) at fixed target ranks.

    python -m paper_2308_01480_gb300.accuracy_study e2 --ranks 2-11
    python -m paper_2308_01480_gb300.accuracy_study e6 --ranks 2-11 --snr 5
    python -m paper_2308_01480_gb300.accuracy_study e6 --ranks 5 --snr 0,5,10,15,20
    python -m paper_2308_01480_gb300.accuracy_study e1 --ranks 5,10,15,20,25,30

e1: 500^3 decaying-spectrum tensor; e2: 45^5 power function (h = 5); e6: e2
with white noise at a measured SNR (dB).  p = 2, q = 2, FP32 storage.
Randomized methods run as one CUDA graph per decomposition (the mean of
three timed launches after one warm-up); TT-SVD is host-synchronous per
mode.  The relative error and the PSNR (Sec. 4: N ||A_hat||_max^2 /
||A - A_hat||_F^2, N the number of entries) are evaluated on the GPU in
float64 against the float64 tensor.  Prints one JSON line per run and a
markdown table.
"""
import argparse
import json
import sys

import numpy as np

METHODS = ("tt_rbki", "tt_rbki_acc", "tt_rsi", "tt_rsvd", "tt_svd")


def error_and_psnr(A64, cores):
    """(||A - A_hat||_F / ||A||_F, PSNR) on the device in float64; A64 is the
    float64 tensor on the GPU, A_hat the contraction of the cores."""
    import torch
    dims = A64.shape
    M = cores[-1].double().reshape(cores[-1].shape[0], -1)
    for G in reversed(cores[1:-1]):
        ra, I, rb = G.shape
        M = (G.double().reshape(ra * I, rb) @ M).reshape(ra, -1)
    F = cores[0].double().reshape(dims[0], -1)
    Am = A64.reshape(dims[0], -1)
    err2, peak = 0.0, 0.0
    step = max(1, int(2 ** 26 // max(1, Am.shape[1])))
    for s in range(0, dims[0], step):
        Ah = F[s:s + step] @ M
        err2 += float(torch.sum((Am[s:s + step] - Ah) ** 2))
        peak = max(peak, float(torch.max(torch.abs(Ah))))
    eps = float(np.sqrt(err2) / float(torch.linalg.norm(Am)))
    psnr = float(10.0 * np.log10(A64.numel() * peak * peak / err2)) if err2 > 0 else float("inf")
    return eps, psnr


def _time(fn, steps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def run_case(A, ranks, oversample, q, seed, methods=METHODS):
    """Each method on the float64 tensor A (decomposed in FP32) at the given
    ranks: {method: {"ms": ..., "eps": ..., "psnr": ..., "ranks": [...]}}."""
    import torch
    import paper_2308_01480_gb300 as tt
    t32 = torch.from_numpy(A.astype(np.float32)).cuda()
    A64 = torch.from_numpy(A).cuda()
    out = {}
    for name in methods:
        if name == "tt_svd":
            holder = {}

            def step():
                holder["cores"], holder["rr"] = tt.tt_svd(t32, eps=0.0, max_ranks=ranks)

            ms = _time(step)
            cores, rr = holder["cores"], holder["rr"]
        else:
            method = tt.TT_METHOD_RSI if name == "tt_rsi" else tt.TT_METHOD_RBKI
            qm = 0 if name == "tt_rsvd" else q
            pb = tt.Problem(t32, ranks, oversample, qm, seed)
            g = tt.BatchGraph([pb], tt.options(storage=tt.TT_F32, method=method,
                                               accurate_rr=(name == "tt_rbki_acc")))
            ms = _time(g.launch)
            if g.device_status() != [0]:
                raise RuntimeError(f"{name}: device status not OK")
            g.close()
            cores, rr = pb.cores, pb.rr
        eps, psnr = error_and_psnr(A64, cores)
        out[name] = {"ms": ms, "eps": eps, "psnr": psnr, "ranks": list(rr)}
    del t32, A64
    torch.cuda.empty_cache()
    return out


def _ints(text):
    vals = []
    for part in text.split(","):
        if "-" in part:
            a, b = part.split("-")
            vals += list(range(int(a), int(b) + 1))
        else:
            vals.append(int(part))
    return vals


def main(argv):
    from paper_2308_01480_gb300 import workloads as W
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("experiment", choices=["e1", "e2", "e6"])
    ap.add_argument("--ranks", default="2-11")
    ap.add_argument("--snr", default="5")
    ap.add_argument("--q", type=int, default=2)
    args = ap.parse_args(argv)
    snrs = [float(x) for x in args.snr.split(",")] if args.experiment == "e6" else [None]
    rows = []
    for snr in snrs:
        base = None
        for r in _ints(args.ranks):
            w = W.study_workload(args.experiment, r, snr if snr is not None else 5.0, args.q)
            if base is None:
                base = W.make_tensor(w)      # the tensor does not depend on r
            res = run_case(base, w.ranks, w.oversample, w.q, w.omega_seed)
            row = {"experiment": args.experiment, "workload": w.name, "rank": r, "snr_db": snr,
                   "p": w.oversample, "q": w.q, "results": res}
            print(json.dumps(row), flush=True)
            rows.append(row)
    print("\n| workload | r | " + " | ".join(f"{m} ms / eps / PSNR" for m in METHODS) + " |")
    print("|---|---:|" + "---:|" * len(METHODS))
    for row in rows:
        cells = [f"{row['results'][m]['ms']:.2f} / {row['results'][m]['eps']:.3e} / {row['results'][m]['psnr']:.1f}"
                 for m in METHODS]
        print(f"| {row['workload']} | {row['rank']} | " + " | ".join(cells) + " |")


if __name__ == "__main__":
    main(sys.argv[1:])
