"""The C-ABI library: loads without a GPU, exports every declared entry
point, its header is plain C that a C program links against, and its
quadrant-index table (the block tags of Sec. III-B) encodes
Strassen's identity at every depth.  No kernel runs here."""
import itertools
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_in_header():
    with open(os.path.join(ROOT, "include", "stark.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^STARK_API\s+[\w\s\*]*?\b(stark_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_in_header()
    assert "stark_plan" in names and "stark_mul" in names and len(names) >= 10


def test_library_exports_every_declared_symbol(stark_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", stark_lib.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(stark_\w+)", out))
    missing = [n for n in declared_in_header() if n not in exported]
    assert not missing, missing
    # and the binding only calls declared entry points
    assert set(stark_lib.declared_symbols()) <= set(declared_in_header())


def test_strerror_and_codes(stark_lib):
    for s in stark_lib.Status:
        assert isinstance(stark_lib.strerror(s), str) and stark_lib.strerror(s)


U = np.array([[1, 0, 0, 1], [0, 0, 1, 1], [1, 0, 0, 0], [0, 0, 0, 1],
              [1, 1, 0, 0], [-1, 0, 1, 0], [0, 1, 0, -1]])


def dense(stark_lib, depth, side):
    count, quad, sign = stark_lib.quadrant_table(depth, side)
    P, Q = 7 ** depth, 4 ** depth
    T = np.zeros((P, Q), np.int64)
    for l in range(P):
        for t in range(count[l]):
            assert T[l, quad[l, t]] == 0  # no quadrant listed twice
            T[l, quad[l, t]] = sign[l, t]
    return T, count


@pytest.mark.parametrize("depth", [0, 1, 2, 3])
def test_table_satisfies_brent_equations(stark_lib, depth):
    # sum_l W[c,l] U[l,a] V[l,b] = [A_a B_b contributes to C_c] for d-level
    # quadrant paths (a, b, c): the table reproduces the classical product.
    Ut, cu = dense(stark_lib, depth, 0)
    Vt, cv = dense(stark_lib, depth, 1)
    Wt, cw = dense(stark_lib, depth, 2)
    Q = 4 ** depth
    got = np.einsum("lc,la,lb->abc", Wt, Ut, Vt)

    def rc(q):
        r = c = 0
        for k in range(depth):
            digit = (q >> (2 * (depth - 1 - k))) & 3
            r = 2 * r + (digit >> 1)
            c = 2 * c + (digit & 1)
        return r, c

    want = np.zeros((Q, Q, Q), np.int64)
    for a, b in itertools.product(range(Q), repeat=2):
        (ai, aj), (bj, bk) = rc(a), rc(b)
        if aj == bj:
            c = [q for q in range(Q) if rc(q) == (ai, bk)][0]
            want[a, b, c] = 1
    assert np.array_equal(got, want)
    # 12^d nonzeros per operand and per combine table, at most 2^d per leaf
    for cnt in (cu, cv, cw):
        assert cnt.sum() == 12 ** depth and cnt.max() <= 2 ** depth


def test_table_level1_is_alg1(stark_lib):
    Ut, _ = dense(stark_lib, 1, 0)
    assert np.array_equal(Ut, U)


def test_table_rejects_bad_depth(stark_lib):
    with pytest.raises(stark_lib.StarkError):
        stark_lib.quadrant_table(5, 0)


def test_header_is_plain_c_and_links(stark_lib, tmp_path):
    """include/stark.h compiles as pedantic C99 and a C program links
    libstark.so and calls its host-only entry points."""
    import shutil
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    lib = stark_lib.library_path()
    exe = str(tmp_path / "abi_client")
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_client.c"), "-o", exe, lib,
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split(maxsplit=12)
    # C targets per product at depth 1: M1 -> C11, C22; M2 -> C21, C22; M3 -> C12, C22;
    # M4 -> C11, C21; M5 -> C11, C12; M6 -> C22; M7 -> C11
    assert out[0] == "0" and [int(v) for v in out[1:8]] == [2, 2, 2, 2, 2, 1, 1]
    status, depth, levels, nbytes = (int(v) for v in out[8:12])
    assert status == 0 and levels == 0 and 0 <= depth <= 4
    g = (1 << depth) * 64
    npad = -(-1024 // g) * g
    assert nbytes == 2 * 7 ** depth * (npad >> depth) ** 2 * 8 + (1 << 20)
    assert out[12].strip() == stark_lib.strerror(stark_lib.Status.ENOMEM)
