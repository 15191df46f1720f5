"""Admission of the request server, on the host (no GPU): which recursion
depth and workspace traversal a request of side n gets under a device-memory
budget, and the bytes counted for it.  The workspace holds the leaf operand
planes of the 7^d leaves of side L = n_pad / 2^d (Sec. III-B, Alg. 1 applied d
times), or one subtree's share of them when the top levels are traversed
depth first (7^levels subtrees, one at a time)."""
import pytest

MIB = 1 << 20
SPLIT = ("F32_SPLIT_BF16", "F32_SPLIT_TF32")


def operands(dtype, n, d):
    """Operand-plane bytes and n_pad at depth d: n padded to a multiple of
    2^d x the leaf tile granule (128 for the split dtypes, 64 otherwise);
    per element hi + lo bf16 (4 B), hi + lo tf32 or one 8-byte value."""
    g = (1 << d) * (128 if dtype in SPLIT else 64)
    npad = max(g, -(-n // g) * g)
    L = npad >> d
    per = 4 if dtype == "F32_SPLIT_BF16" else 8
    return 2 * 7 ** d * L * L * per, npad


def expected_bytes(dtype, n, d, levels, staged=False):
    ops, npad = operands(dtype, n, d)
    stage = npad * npad * 4 if staged and dtype in SPLIT else 0
    return ops // 7 ** levels + MIB + stage


def traversals(dtype, d):
    """Depth-first levels a workspace of depth d may take: the subtree
    loaders cover depth <= 3, two levels only for the split dtypes."""
    out = [0]
    if 1 <= d <= 3:
        out.append(1)
        if d >= 2 and dtype in SPLIT:
            out.append(2)
    return out


def query(S, budget, n, dtype, staged=False):
    return S.server_admission(budget, n, getattr(S.DType, dtype), staged)


CASES = [("F32_SPLIT_BF16", 16384), ("F32_SPLIT_BF16", 4096), ("F32_SPLIT_BF16", 1000),
         ("F32_SPLIT_TF32", 3000), ("F64", 1024), ("F64", 777), ("I64", 2048), ("I64", 4096)]


@pytest.mark.parametrize("dtype,n", CASES)
def test_ample_budget_is_breadth_first(stark_lib, dtype, n):
    a = query(stark_lib, 1 << 50, n, dtype)
    assert 0 <= a["depth"] <= 4 and a["levels"] == 0
    assert a["bytes"] == expected_bytes(dtype, n, a["depth"], 0)


@pytest.mark.parametrize("dtype,n", [c for c in CASES if c[0] in SPLIT])
def test_staged_c_adds_its_copy(stark_lib, dtype, n):
    a = query(stark_lib, 1 << 50, n, dtype, staged=True)
    assert a["bytes"] == expected_bytes(dtype, n, a["depth"], 0, staged=True)
    # not for the plain dtypes, whose combine never stages C
    b = query(stark_lib, 1 << 50, n, "F64", staged=True)
    assert b["bytes"] == expected_bytes("F64", n, b["depth"], 0)


@pytest.mark.parametrize("dtype,n", CASES)
def test_budget_sweep_follows_the_admission_rule(stark_lib, dtype, n):
    """At every budget: the first choice's depth with the fewest depth-first
    levels that fit, else some other depth whose workspace fits, else ENOMEM
    exactly when no (depth, levels) pair fits at all."""
    S = stark_lib
    first = query(S, 1 << 50, n, dtype)["depth"]
    options = {(d, l): expected_bytes(dtype, n, d, l) for d in range(5) for l in traversals(dtype, d)}
    budgets = sorted(set(options.values()) | {b - 1 for b in options.values()} | {MIB, 1 << 50})
    for budget in budgets:
        fitting = {k for k, v in options.items() if v <= budget}
        if not fitting:
            with pytest.raises(S.StarkError) as e:
                query(S, budget, n, dtype)
            assert e.value.status == S.Status.ENOMEM
            continue
        a = query(S, budget, n, dtype)
        key = (a["depth"], a["levels"])
        assert key in fitting and a["bytes"] == options[key], (budget, a)
        at_first = sorted(l for d, l in fitting if d == first)
        if at_first:
            assert key == (first, at_first[0]), (budget, a)


def test_depth_first_shrinks_the_workspace_sevenfold_per_level(stark_lib):
    # 3xBF16 at n = 16384: the breadth-first workspace, then one and two
    # levels depth first at the same depth as the budget tightens
    S = stark_lib
    a0 = query(S, 1 << 50, 16384, "F32_SPLIT_BF16")
    d = a0["depth"]
    assert 2 <= d <= 3
    a1 = query(S, a0["bytes"] - 1, 16384, "F32_SPLIT_BF16")
    assert (a1["depth"], a1["levels"]) == (d, 1)
    assert a1["bytes"] - MIB == (a0["bytes"] - MIB) // 7
    a2 = query(S, a1["bytes"] - 1, 16384, "F32_SPLIT_BF16")
    assert (a2["depth"], a2["levels"]) == (d, 2)
    assert a2["bytes"] - MIB == (a0["bytes"] - MIB) // 49


def test_fp64_budget_for_one_depth1_subtree(stark_lib):
    # the budget of the GPU server test: side 1024 in FP64 fits only as one
    # depth-1 subtree (2 x 512^2 x 8 B = 4 MiB, + 1 MiB for the tables)
    a = query(stark_lib, (5 << 20) + (512 << 10), 1024, "F64")
    assert (a["depth"], a["levels"], a["bytes"]) == (1, 1, 5 << 20)
    with pytest.raises(stark_lib.StarkError) as e:
        query(stark_lib, (5 << 20) + (512 << 10), 2048, "F64")
    assert e.value.status == stark_lib.Status.ENOMEM


def test_rejects_bad_arguments(stark_lib):
    S = stark_lib
    for n in (-1, (1 << 20) + 1):
        with pytest.raises(S.StarkError) as e:
            S.server_admission(1 << 30, n, S.DType.F64)
        assert e.value.status == S.Status.EINVAL
    assert S._lib.stark_server_admission(1 << 30, 64, 9, 0, None, None, None) == S.Status.EINVAL  # no dtype 9
    # an empty product still takes its (smallest) workspace
    assert query(S, 1 << 30, 0, "F64")["bytes"] > 0
