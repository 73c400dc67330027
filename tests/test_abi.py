"""CPU-side checks of the boundary: the library builds for sm_103a, loads,
and exports every entry point declared in include/*.h (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(receipt_[a-z_0-9]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2010_08695_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("receipt_build_csr", "receipt_count_butterflies", "receipt_tip_decompose",
              "receipt_decompose_batch", "receipt_get_stats", "receipt_last_error",
              "receipt_graph_destroy", "receipt_tip_decompose_host"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_symbols_are_c_linkage(lib):
    from paper_2010_08695_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (receipt_\w+)", out))
    assert _declared() <= exported


def test_options_default_and_last_error_without_gpu(lib):
    import paper_2010_08695_gb300 as R
    o = R.Options()
    lib.receipt_options_default(ctypes.byref(o))
    assert o.P == 150 and o.n_bounds == 0 and o.timing == 0
    lib.receipt_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.receipt_last_error(), bytes)


def test_round_launch_modes_marshal_without_gpu(lib):
    # Python's round_graphs: False -> 0 (device-driven rounds, the default),
    # True -> 1 (one graph launch per round), -1 -> -1 (separate launches)
    import paper_2010_08695_gb300 as R
    assert R._options(round_graphs=False)[0].round_graphs == 0
    assert R._options(round_graphs=True)[0].round_graphs == 1
    assert R._options(round_graphs=-1)[0].round_graphs == -1
    o = R.Options()
    lib.receipt_options_default(ctypes.byref(o))
    assert o.round_graphs == 0


def test_null_arguments_are_rejected_without_gpu(lib):
    import paper_2010_08695_gb300 as R
    R.load()
    # null output handle / null graph: validated before any CUDA call
    assert lib.receipt_build_csr(None, None, 0, 1, 1, 1, None, None) == 1
    assert lib.receipt_get_stats(None, None) == 1
    assert lib.receipt_graph_info(None, None, None, None) == 1
    assert lib.receipt_graph_destroy(None) == 0


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes mirror of a header struct has the C size and the C offset
    of each field (checked with offsetof in a program gcc builds from
    include/receipt.h)."""
    import shutil
    import paper_2010_08695_gb300 as R
    if not shutil.which("gcc"):
        pytest.skip("gcc not found")
    pairs = [(R.Options, "receipt_options"), (R.Stats, "receipt_stats"),
             (R.Round, "receipt_round"), (R.Subset, "receipt_subset"),
             (R.ServerConfig, "receipt_server_config"), (R.ServerStats, "receipt_server_stats")]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "receipt.h"',
             "int main(void) {"]
    want = []
    for cls, cname in pairs:
        lines.append(f'    printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(cls, f).offset)
    lines += ["    return 0;", "}"]
    src = str(tmp_path / "layout_probe.c")
    exe = str(tmp_path / "layout_probe")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
    got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got == want


def test_support_bound_without_gpu():
    """The count bound behind RECEIPT_ERR_OVERFLOW (host arithmetic): it
    holds on random graphs against the oracle's counts, is exact for the
    U side of K_{a,b}, and reports overflow once it reaches 2^63."""
    import numpy as np
    import oracle
    import paper_2010_08695_gb300 as R
    import synth
    for seed in range(40):
        rng = np.random.default_rng(seed)
        nu, nv = int(rng.integers(2, 40)), int(rng.integers(2, 40))
        eu, ev = synth.random_small(nu, nv, float(rng.uniform(0.05, 0.9)), seed)
        if len(eu) == 0:
            continue
        cu, cv = oracle.count_2hop(eu, ev, nu, nv)
        du = np.bincount(eu, minlength=nu)
        dv = np.bincount(ev, minlength=nv)
        assert int(cu.max()) <= R.receipt_support_bound(nu, du.max(), dv.max(), len(eu))
        assert int(cv.max()) <= R.receipt_support_bound(nv, dv.max(), du.max(), len(eu))
    for a, b in ((2, 2), (5, 3), (7, 11), (30, 4)):
        eu, ev = synth.complete_bipartite(a, b)
        cu, _ = oracle.count_2hop(eu, ev, a, b)
        assert R.receipt_support_bound(a, b, a, a * b) == int(cu.max()) == (a - 1) * b * (b - 1) // 2
    # the library's own limits (m < 2^31) keep every count below 2^61
    big = 2 ** 31 - 1
    assert R.receipt_support_bound(big, big, big, big - 1) < 2 ** 61
    with pytest.raises(R.ReceiptError) as ei:
        R.receipt_support_bound(big, big, big, 2 ** 40)
    assert ei.value.status == 5
    with pytest.raises(R.ReceiptError) as ei:
        R.receipt_support_bound(-1, 1, 1, 1)
    assert ei.value.status == 1
