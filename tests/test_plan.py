"""The planner's per-mode routes, queried through the C ABI on CPU.

tt_rbki_plan_modes reports the plan tt_rbki_decompose follows; these tests
pin its rules on the benchmark's 40^5 workload and on small cases: the
Krylov dimension cap of Alg. 3 (the basis stops at D = min(m, n) columns),
the two exhaustion routes, the Gram-power route and its switch, Alg. 4's
power count, and which passes run on the tensor cores.
"""
import os

import pytest

import paper_2308_01480_gb300 as tt
from paper_2308_01480_gb300 import _native as N
from paper_2308_01480_gb300 import build as B

DIMS = (40, 40, 40, 40, 40)
RANKS = (20, 20, 20, 20)


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not os.path.exists(N.LIB_PATH):
        B.build()
    return N.lib()


def bf16(**kw):
    return tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16, **kw)


def test_benchmark_workload_routes():
    modes = tt.plan_modes(DIMS, RANKS, 10, 4, bf16())
    assert [(e["m"], e["n"]) for e in modes] == [(40, 2560000), (800, 64000), (800, 1600), (800, 40)]
    assert [e["route"] for e in modes] == ["gram_rows", "gram_power", "gram_power", "gram_cols"]
    # b = 30; the mode-1 basis stops at D = 40 after two blocks, mode 4 at D = n = 40
    assert [e["b"] for e in modes] == [30] * 4
    assert [e["basis_cols"] for e in modes] == [40, 150, 150, 40]
    assert [e["blocks"] for e in modes] == [2, 5, 5, 2]
    assert [e["powers"] for e in modes] == [0, 5, 5, 0]
    assert [e["tensor_cores"] for e in modes] == [True, True, True, False]   # n = 40 < 64 at mode 4
    assert [e["r_in"] for e in modes] == [1, 20, 20, 20] and [e["r_out"] for e in modes] == [20] * 4


def test_switches_fall_back_to_streaming():
    modes = tt.plan_modes(DIMS, RANKS, 10, 4, bf16(gram_power=False))
    assert [e["route"] for e in modes] == ["gram_rows", "krylov", "krylov", "gram_cols"]
    modes = tt.plan_modes(DIMS, RANKS, 10, 4, bf16(exhaust_gram=False))
    # mode 1: two powers over n = 2.56M columns, too few for the BF16 Gram-power rule;
    # mode 4: two powers over an 800 x 40 unfolding take it
    assert [e["route"] for e in modes] == ["krylov", "gram_power", "gram_power", "gram_power"]
    assert modes[0]["powers"] == 2 and modes[0]["fused_power"]


def test_fp32_storage_streams_on_simt():
    modes = tt.plan_modes(DIMS, RANKS, 10, 4, tt.options())
    assert not any(e["tensor_cores"] for e in modes)
    # FP32 has no tensor-core Gram: mode 2 (n = 64,000 > 8192) streams its powers
    assert [e["route"] for e in modes] == ["gram_rows", "krylov", "gram_power", "gram_cols"]


def test_subspace_iteration_counts():
    modes = tt.plan_modes((30, 20, 50), (4, 6), 2, 3, tt.options(method=tt.TT_METHOD_RSI, exhaust_gram=False))
    assert [e["blocks"] for e in modes] == [1, 1]
    assert [e["basis_cols"] for e in modes] == [6, 8]
    assert [e["powers"] for e in modes] == [4, 4]      # q powers plus the one that feeds Rayleigh-Ritz


def test_q_zero_is_a_single_sketch():
    modes = tt.plan_modes((30, 20, 50), (4, 6), 2, 0, tt.options(exhaust_gram=False, gram_power=False))
    assert [e["blocks"] for e in modes] == [1, 1] and [e["powers"] for e in modes] == [1, 1]
    assert [e["route"] for e in modes] == ["krylov", "krylov"]


def test_rank_clamp_shows_in_plan():
    modes = tt.plan_modes((3, 5, 4), (9, 9), 1, 1, tt.options())
    assert [(e["r_in"], e["r_out"]) for e in modes] == [(1, 3), (3, 4)]
    assert [(e["m"], e["n"]) for e in modes] == [(3, 20), (15, 4)]


def test_argument_errors():
    with pytest.raises(tt.TTError):
        tt.plan_modes((4,), (), 1, 1)
    arr = (N.TTModePlan * 1)()
    assert N.lib().tt_rbki_plan_modes(N.i64_array(DIMS), 5, N.i64_array(RANKS), 10, 4, None, arr, 1) == N.TT_EINVAL
    assert N.lib().tt_rbki_plan_modes(N.i64_array(DIMS), 5, N.i64_array(RANKS), 10, 4, None, None, 4) == N.TT_EINVAL


def test_bench_plan_summary():
    import bench
    from paper_2308_01480_gb300 import workloads as W
    w = W.CONFIGS[bench.CONFIG_ID]
    got = bench.plan_summary(tt, w, bf16())
    assert got == ["40x2560000 gram_rows tc", "800x64000 gram_power tc", "800x1600 gram_power tc",
                   "800x40 gram_cols"]


def test_bench_family_names_exist_in_the_library():
    """The kernel families bench.py reads (DRAM traffic, library GEMMs) are
    names the library's launch accounting actually records."""
    import glob
    import re
    import bench
    src = "".join(open(f).read() for f in glob.glob(os.path.join(os.path.dirname(N.__file__), "csrc", "*.cu")))
    names = set(re.findall(r'ProfScope \w+\("(\w+)"', src))
    assert set(bench.NCU_TRAFFIC) <= names
    assert set(bench.LIBRARY_FAMILIES) <= names


def test_literal_plan_counts_powers():
    """paper_literal: r_k columns, one power for Alg. 3 (q >= 1), none for
    q = 0, q powers for Alg. 4; never an exhaustion Gram route."""
    dims, ranks = (40, 40, 40, 40, 40), (20, 20, 20, 20)
    for method, q, want in ((tt.TT_METHOD_RBKI, 4, 1), (tt.TT_METHOD_RBKI, 0, 0), (tt.TT_METHOD_RSI, 3, 3)):
        modes = tt.plan_modes(dims, ranks, 10, q, tt.options(storage=tt.TT_BF16, method=method, paper_literal=True))
        assert all(e["powers"] == want and e["basis_cols"] == e["r_out"] for e in modes)
        assert all(e["route"] in ("krylov", "gram_power") for e in modes)


def test_bench_algorithmic_bytes_per_decomposition():
    """The roofline numerator bench.py reports: per mode, (q_eff + 2) reads of
    the unfolding (sketch, q_eff Krylov steps, projection), one read of Omega
    and one write of the remainder, q_eff capped by the Krylov dimension.
    For the 40^5 workload by hand (entries): mode 1 40 x 2,560,000, q_eff 1:
    3 * 102.4M + 30 * 2.56M + 20 * 2.56M = 435.2M; mode 2 800 x 64,000,
    q_eff 4: 6 * 51.2M + 50 * 64,000 = 310.4M; mode 3 800 x 1,600: 7.76M;
    mode 4 800 x 40, q_eff 1: 98,000; in all 753.458M entries, 1506.916 MB
    in BF16.  The other two single-GPU workloads likewise."""
    import bench
    from paper_2308_01480_gb300 import workloads as W
    want = {(3, 2): 1506.916e6, (3, 4): 3013.832e6, (4, 2): 1573.40096e6, (4, 4): 3146.80192e6,
            (2, 4): 861.543552e6, (2, 2): 430.771776e6}
    for (cfg, e), nbytes in want.items():
        code = tt.TT_BF16 if e == 2 else tt.TT_F32
        got = bench.algorithmic_bytes(tt, W.CONFIGS[cfg], tt.options(storage=code, remainder=code), e)
        assert got == pytest.approx(nbytes, rel=1e-12), (cfg, e, got)
