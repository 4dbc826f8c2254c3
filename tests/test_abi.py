"""CPU-side checks of the boundary: the library builds, loads and exports
every symbol the public header declares; host-only entry points behave; no
kernel is launched."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1701_03512_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bt():
    from paper_1701_03512_gb300 import build as b
    b.build()
    from paper_1701_03512_gb300 import btree
    btree.lib()
    return btree


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(bt_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("bt_create", "bt_destroy", "bt_price_exact", "bt_exact_plan_run", "bt_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(bt):
    L = ctypes.CDLL(bt.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layout(bt):
    assert ctypes.sizeof(bt.bt_option) == 80
    assert ctypes.sizeof(bt.bt_result) == 40


def test_status_strings(bt):
    L = bt.lib()
    assert L.bt_status_str(0) == b"BT_OK"
    assert L.bt_status_str(3) == b"BT_EBUDGET"
    assert b"sm_103a" in L.bt_version()


def test_tree_params_host(bt):
    """bt_tree_params runs on the host; it agrees with the oracle's tree."""
    from oracle import py_oracle as O
    for kind in (W.TREE_CRR, W.TREE_SEYDEL):
        o = W.opt(32, 20.0, 100.0, 0.06, 3.0, 1.0, W.ASIAN_ARITH_PUT, kind)
        u, d, p = bt.bt_tree_params(o)
        uo, do, po = O.tree(kind, 32, 3.0, 0.06, 1.0)
        assert (u, d, p) == pytest.approx((uo, do, po), rel=1e-15)


@pytest.mark.parametrize("bad,msg", [
    (dict(S0=-1.0), "S0"), (dict(T=0.0), "T must"), (dict(sigma=0.0), "sigma"),
    (dict(K=float("nan")), "non-finite"), (dict(payoff=9), "payoff"), (dict(tree_kind=7), "tree_kind"),
    (dict(sigma=0.001, rate=0.5), "not in (0,1)"),
])
def test_tree_params_rejects(bt, bad, msg):
    o = dict(W.opt(20, 100.0, 100.0, 0.05, 0.2, 1.0, W.ASIAN_ARITH_CALL), **bad)
    with pytest.raises(bt.BtError) as e:
        bt.bt_tree_params(o)
    assert e.value.status == bt.BT_EINVAL and msg in str(e.value)


def test_explicit_tree_needs_ud_one(bt):
    o = W.opt(5, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL, W.TREE_EXPLICIT, u=1.1, d=0.9, p=0.5)
    with pytest.raises(bt.BtError):
        bt.bt_tree_params(o)
    o = W.opt(5, 100.0, 100.0, 0.0, 0.2, 1.0, W.EURO_CALL, W.TREE_EXPLICIT, u=1.1, d=1 / 1.1, p=0.5)
    assert bt.bt_tree_params(o) == (1.1, 1 / 1.1, 0.5)


def test_create_without_gpu_fails_cleanly(bt):
    """No GPU in this container: bt_create must fail with BT_ECUDA, not crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bt.BtError) as e:
        bt.bt_create(0)
    assert e.value.status == bt.BT_ECUDA


def test_options_array_roundtrip(bt):
    opts = W.batched_exact_workload(32, 0, 4)
    a = bt.options_array(opts)
    assert a.shape == (8,) and a["N"].tolist() == [32] * 8
    assert a["payoff"].tolist() == [2, 3] * 4
    assert np.allclose(a["S0"][::2], W.option_sets(0, 4)["S0"])


def test_exact_split_needs_no_device(bt):
    """The pass's prefix/suffix split (Section 3's rank bits as the prefix),
    queried on the host: L = N - 15 (at least 1, at most 13) suffix steps, so
    an option keeps 2^5 work items of 2^10 prefixes where it can, and
    L = N - 17 for the FP64 pass (2^7 items); FP32 arithmetic Asians up to
    N = 27 sum each suffix as a class, with at most 12."""
    cases = [  # (N, payoff, precision) -> (P, L)
        ((36, W.ASIAN_ARITH_CALL, bt.BT_PREC_FP32_COMP), (23, 13)),
        ((28, W.ASIAN_ARITH_PUT, bt.BT_PREC_FP32_COMP), (15, 13)),
        ((27, W.ASIAN_ARITH_PUT, bt.BT_PREC_FP32_COMP), (15, 12)),
        ((26, W.ASIAN_ARITH_PUT, bt.BT_PREC_FP64), (17, 9)),
        ((30, W.ASIAN_ARITH_PUT, bt.BT_PREC_FP64), (17, 13)),
        ((30, W.ASIAN_GEO_CALL, bt.BT_PREC_FP32_COMP), (17, 13)),
        ((20, W.ASIAN_ARITH_CALL, bt.BT_PREC_FP64), (17, 3)),
        ((5, W.EURO_PUT, bt.BT_PREC_FP64), (4, 1)),
    ]
    for (N, pay, prec), (P, L) in cases:
        sp = bt.bt_exact_split(W.opt(N, 100.0, 100.0, 0.05, 0.2, 1.0, pay), prec)
        assert (sp["P"], sp["L"]) == (P, L), (N, pay, prec, sp)
        assert sp["prefixes_per_item"] == 1024
        assert sp["n_items"] == max(1, (1 << P) // 1024)
    with pytest.raises(bt.BtError) as e:
        bt.bt_exact_split(W.opt(41, 100.0, 100.0, 0.05, 0.2, 1.0, W.EURO_CALL))
    assert e.value.status == bt.BT_EINVAL


def test_skewed_trees_route_to_the_class_pass(bt):
    """Host routing of FP32_COMP: an arithmetic Asian from 2^28 paths keeps
    the per-path pass (L = 13) only while the tree has at least 2^27
    effective paths, (p^2 + (1-p)^2)^-N; below that the pair-sum class pass
    (L <= 12). FP64 and the other payoffs are unaffected."""
    u = 1.05
    for N in (28, 36):
        pc = 0.5 * (1.0 + math.sqrt(2.0 * 2.0 ** (-27.0 / N) - 1.0))
        for p, L in ((0.5, 13), (pc - 1e-3, 13), (pc + 1e-3, 12), (1 - pc - 1e-3, 12), (1 - pc + 1e-3, 13),
                     (0.996, 12)):
            o = W.opt(N, 100.0, 100.0, 0.0, 0.2, 1.0, W.ASIAN_ARITH_CALL, W.TREE_EXPLICIT, u=u, d=1 / u, p=p)
            assert bt.bt_exact_split(o, bt.BT_PREC_FP32_COMP)["L"] == L, (N, p)
            assert bt.bt_exact_split(o, bt.BT_PREC_FP64)["L"] == min(13, N - 17)
            g = dict(o, payoff=W.ASIAN_GEO_CALL)
            assert bt.bt_exact_split(g, bt.BT_PREC_FP32_COMP)["L"] == 13


def test_plain_c_client(bt, tmp_path):
    """tests/abi_client.c built with gcc against include/btree.h and linked
    to lib/libbtree.so: the boundary from C, no Python in between."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(bt.LIB_PATH)
    exe = str(tmp_path / "abi_client")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(root, "tests", "abi_client.c"), "-L", libdir, "-lbtree",
                    "-Wl,-rpath," + libdir, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "split P=17 L=3" in r.stdout   # FP64 at N=20: 2^7 work items of 2^10 prefixes
