"""Small, fixed invocations of the library for profiling one kernel at a
time (each runs its case three times, so that a profiler told to skip the
first launches of a kernel sees a warm third one):

    python -m paper_2308_01480_gb300.profile_cases pass ga 800 64000 30
        one streaming pass (gram | proj | proj_bf16 | cs | ga) over a seeded
        BF16 m x n unfolding, b columns (proj_bf16: BF16 output, as the
        decomposition writes its remainders)
    python -m paper_2308_01480_gb300.profile_cases eig 150 20
        the Rayleigh-Ritz eigensolver on a k x k PSD matrix, top r
    python -m paper_2308_01480_gb300.profile_cases decompose 3
        full BF16 decompositions of a benchmark workload configuration

Only the public binding is used; inputs are seeded and synthetic.
"""
import sys

import numpy as np


def _pass(op, m, n, b):
    import torch
    import paper_2308_01480_gb300 as tt
    g = torch.Generator(device="cuda").manual_seed(1)
    C = torch.randn(m, n, device="cuda", generator=g).to(torch.bfloat16)
    code = {"gram": tt.TT_PASS_GRAM, "proj": tt.TT_PASS_PROJECT, "proj_bf16": tt.TT_PASS_PROJECT,
            "cs": tt.TT_PASS_SKETCH, "ga": tt.TT_PASS_GRAMAPPLY}[op]
    x = None
    if op == "cs":
        x = torch.randn(n, b, device="cuda", generator=g)
    elif op in ("proj", "proj_bf16", "ga"):
        x = torch.randn(m, b, device="cuda", generator=g)
    ws = torch.empty(tt.pass_workspace_size(code, m, n, b, tt.TT_BF16), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        y = tt.tt_pass(code, C, x=x, workspace=ws, y_dtype=torch.bfloat16 if op == "proj_bf16" else None)
    torch.cuda.synchronize()
    print(op, m, n, b, float(y.float().abs().sum()))


def _eig(k, r):
    import torch
    import paper_2308_01480_gb300 as tt
    rng = np.random.default_rng(k)
    B = rng.standard_normal((k, 4 * k)) * (0.9 ** np.arange(k))[:, None]
    H = torch.from_numpy((B @ B.T).astype(np.float32)).cuda()
    for _ in range(3):
        V, ev = tt.sym_eig_top(H, r)
    torch.cuda.synchronize()
    print(k, r, float(ev.sum()))


def _decompose(config):
    import torch
    import paper_2308_01480_gb300 as tt
    from paper_2308_01480_gb300 import workloads as W
    w = W.CONFIGS[config]
    A = W.make_tensor(w)
    t = tt.permute_convert(torch.from_numpy(A.astype(np.float32)).cuda(), dst_dtype=torch.bfloat16)
    opts = tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16)
    for _ in range(3):
        cores, rr = tt.decompose(t, w.ranks, w.oversample, w.q, omega_seed=w.omega_seed, opts=opts)
    torch.cuda.synchronize()
    print(rr, float(sum(c.float().abs().sum() for c in cores)))


def main(argv):
    if argv[:1] == ["pass"] and len(argv) == 5:
        _pass(argv[1], int(argv[2]), int(argv[3]), int(argv[4]))
    elif argv[:1] == ["eig"] and len(argv) == 3:
        _eig(int(argv[1]), int(argv[2]))
    elif argv[:1] == ["decompose"] and len(argv) == 2:
        _decompose(int(argv[1]))
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
