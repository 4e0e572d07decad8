"""CPU-only checks of the boundary and host logic: the C-ABI library builds,
loads and exports every symbol include/fnt.h declares (no compute calls), the
binding covers them, and the multi-rank timing reduction of bench.py works
across world_size-2 gloo ranks."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                names += re.findall(r"FNT_API[^;(]*?\b(fnt_\w+)\s*\(", fh.read())
    return sorted(set(names))


@pytest.fixture(scope="module")
def libfnt():
    import paper_2405_04253_gb300 as fnt
    path = fnt.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("fnt_plan_create", "fnt_cdc_run", "fnt_aeq_run", "fnt_cdc_aeq_run", "fnt_session_submit",
                 "fnt_session_poll"):
        assert must in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libfnt):
    missing = [n for n in header_functions() if not hasattr(libfnt, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2405_04253_gb300 as fnt
    assert sorted(fnt.SIGNATURES) == header_functions()


def _c_layout(struct: str, fields) -> dict:
    """sizeof and offsetof of a struct of include/fnt.h, compiled by the host C
    compiler from the header alone."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "fnt.h"', "int main(void) {",
           f'  printf("size %zu\\n", sizeof({struct}));']
    src += [f'  printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    src += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        with open(c, "w") as fh:
            fh.write("\n".join(src) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_binding_struct_layouts_match_the_header():
    """Every struct the binding passes through the C ABI has the header's size
    and field offsets (ctypes structures and the numpy record types)."""
    import paper_2405_04253_gb300 as fnt
    ctypes_structs = {
        "fnt_plan_desc": (fnt.PlanDesc, None),
        "fnt_frame": (fnt.FrameC, {"in_": "in"}),
        "fnt_frame_batch": (fnt.BatchC, None),
        "fnt_op_counts": (fnt.OpCounts, None),
        "fnt_completion": (fnt.Completion, None),
        "fnt_session_stats": (fnt.SessionStats, None),
    }
    for struct, (cls, rename) in ctypes_structs.items():
        names = [f[0] for f in cls._fields_]
        cnames = [(rename or {}).get(n, n) for n in names]
        lay = _c_layout(struct, cnames)
        assert lay["size"] == ctypes.sizeof(cls), struct
        for n, cn in zip(names, cnames):
            assert lay[cn] == getattr(cls, n).offset, (struct, n)
    for struct, dt, rename in (("fnt_request", fnt.REQUEST_DTYPE, {"in_": "in"}),
                               ("fnt_completion", fnt.COMPLETION_DTYPE, {})):
        cnames = [rename.get(n, n) for n in dt.names]
        lay = _c_layout(struct, cnames)
        assert lay["size"] == dt.itemsize, struct
        for n, cn in zip(dt.names, cnames):
            assert lay[cn] == dt.fields[n][1], (struct, n)


def test_library_is_sm103a_only():
    import importlib
    b = importlib.import_module("paper_2405_04253_gb300.build")
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_defaults_without_gpu(libfnt):
    import paper_2405_04253_gb300 as fnt
    lib = fnt.lib()
    assert lib.fnt_version().decode().startswith("fnt ")
    d = fnt.default_desc()
    assert (d.n_cdc, d.alpha_cdc, d.n_aeq, d.alpha_aeq, d.aeq_taps) == (64, 4080, 32, 2, 16)


def test_plan_setters_reject_a_null_plan_without_gpu(libfnt):
    """Launch knobs validate their arguments on the host (no GPU needed)."""
    libfnt.fnt_plan_set_aeq_occupancy.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    libfnt.fnt_plan_set_launch.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
    assert libfnt.fnt_plan_set_aeq_occupancy(None, 8) == 1        # FNT_ERR_INVALID
    assert libfnt.fnt_plan_set_launch(None, 4, 2) == 1


def test_plan_rejects_invalid_radix_without_gpu():
    # eq. (4) is checked on the host before any device call
    import paper_2405_04253_gb300 as fnt
    with pytest.raises(fnt.FntError) as e:
        fnt.Plan(alpha_cdc=2)
    assert e.value.status == fnt.FNT_ERR_BOUND
    with pytest.raises(fnt.FntError) as e:
        fnt.Plan(n_aeq=32, alpha_aeq=4)            # order 16: alpha^32 = 1 but order != 32
    assert e.value.status == fnt.FNT_ERR_BOUND
    for bad in (-1, 65):                          # update period outside [0, 64]
        with pytest.raises(fnt.FntError) as e:
            fnt.Plan(aeq_update_period=bad)
        assert e.value.status == fnt.FNT_ERR_INVALID
    assert fnt.default_desc().aeq_update_period == 0
    with pytest.raises(fnt.FntError) as e:
        fnt.Plan(aeq_freq_sum=3)
    assert e.value.status == fnt.FNT_ERR_INVALID
    assert fnt.default_desc().aeq_freq_sum == 0


def test_product_package_does_not_import_oracle():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2405_04253_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    txt = fh.read()
                assert "import oracle" not in txt and "fnt_oracle" not in txt, f


def test_oracle_does_not_import_product():
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            with open(os.path.join(ROOT, "oracle", f)) as fh:
                txt = fh.read()
            assert "paper_2405_04253_gb300" not in txt and "fnt.h" not in txt


def test_bench_op_model():
    import bench
    assert bench.butterflies(64) == 192 and bench.butterflies(32) == 80
    # 2 pols x 2 fwd + 2 inv transforms x 192 butterflies x 6 + 2 x 64 products x 3, per 48-sample block
    assert bench.cdc_ops(48, 48) == 2 * (4 * 192 * 6 + 128 * 3)
    assert bench.aeq_ops(48, 64) == 68 * 192 * 6 + 32 * 64 * 3 + 16 * 16 * 48 * 2
    assert bench.alu_peak_ops() == pytest.approx(40.27e12, rel=1e-3)


def _gloo_worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    ms = [3.0, 5.0][rank]
    m = bench.reduce_max(ms)
    q.put((rank, m, bench.aggregate(1000, world, m * 1e-3)))
    dist.destroy_process_group()


def test_multirank_timing_reduction_gloo():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 5.0                                 # slowest rank's time
        assert v == pytest.approx(2 * 1000 / 5e-3 / 1e9)


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_max(1.25) == 1.25
    assert bench.aggregate(2 ** 21, 1, 1e-3) == pytest.approx(2 ** 21 / 1e-3 / 1e9)


def test_tab1_multiplication_counts():
    """Tab. 1: FNT-CDC 8 and FNT-AEQ 64 real multiplications per symbol at the
    paper's operating point (64-point CDC with 50 % overlap, 32-point AEQ).
    The library counts them by running the product-stage templates the
    kernels execute (the CDC's spectral stage, each AEQ kernel's product
    stage) on the host with a counting arithmetic policy, so a product added
    to a kernel's product stage changes these numbers.  The FD / TD rows and
    the complexity reductions of the text are context (evaluated here from
    the table's formulas)."""
    import math
    import paper_2405_04253_gb300 as fnt
    oc = fnt.op_counts(17, cdc_step=32, n_aeq=32, alpha_aeq=2)
    assert oc["cdc_mults_per_symbol"] == 8
    assert oc["aeq_mults_per_symbol"] == 64
    assert oc["aeq_cta_mults_per_symbol"] == 64
    assert fnt.op_counts(17, n_aeq=64, alpha_aeq=4080)["aeq_cta_mults_per_symbol"] == 32 * 64 / 48
    fd_cdc = lambda n: 12 * math.log2(n) + 12
    fd_aeq = lambda n: 24 * math.log2(n) + 32
    assert round(1 - 64 / fd_aeq(32), 2) == 0.58                    # AEQ: -58 %
    assert round(1 - 8 / fd_cdc(32), 2) == 0.89                     # CDC: -89 % (at log2 N = 5)
    assert round(1 - (8 + 64) / (fd_cdc(32) + fd_aeq(32)), 2) == 0.68
    # the default step N - L + 1 spends fewer products per symbol
    assert fnt.op_counts(17)["cdc_mults_per_symbol"] == 128 / 24
    assert fnt.op_counts(17, n_aeq=64, alpha_aeq=4080)["aeq_mults_per_symbol"] == 32 * 64 / 48


def test_request_records_marshal_pointers_and_sizes():
    """fnt.Requests packs (link, in, n, out) into fnt_request records with the
    buffers' addresses and sample counts, and keeps the buffers alive."""
    import numpy as np
    import paper_2405_04253_gb300 as fnt
    xs = [np.zeros((n, 2, 2), np.int8) for n in (5, 0, 1234)]
    outs = [np.zeros((max(1, n // 2), 4), np.int16) for n in (5, 0, 1234)]
    r = fnt.Requests([3, 0, 7], xs, outs)
    assert len(r) == 3 and r.rec.dtype == fnt.REQUEST_DTYPE
    assert r.rec["link"].tolist() == [3, 0, 7]
    assert r.rec["n"].tolist() == [5, 0, 1234]
    assert r.rec["reserved"].tolist() == [0, 0, 0]
    assert r.rec["in_"].tolist() == [x.ctypes.data for x in xs]
    assert r.rec["out"].tolist() == [o.ctypes.data for o in outs]
    assert r.bufs[2][0] is xs[2] and r.bufs[2][1] is outs[2]
    r2 = fnt.Requests([1], xs[:1], outs[:1], ns=[4])
    assert r2.rec["n"].tolist() == [4]


def test_every_entry_point_rejects_null_handles_without_gpu():
    """The ABI never crashes on a null handle: every status-returning call
    returns FNT_ERR_INVALID (destroy calls: FNT_OK), and the counters of a null
    object read as zero, all before any CUDA call."""
    import paper_2405_04253_gb300 as fnt
    L = fnt.lib()
    inv = fnt.FNT_ERR_INVALID
    calls = {
        "fnt_plan_create": (None, None),
        "fnt_op_counts_for": (None, 17, None),
        "fnt_cdc_run": (None, None, None),
        "fnt_aeq_run": (None, None, None),
        "fnt_cdc_aeq_run": (None, None, None),
        "fnt_batch_create": (None, None, 2, 0, None),
        "fnt_batch_launch": (None, None),
        "fnt_batch_set_input_copy": (None, 1),
        "fnt_batch_launch_stage": (None, 0, None),
        "fnt_plan_set_launch": (None, 4, 2),
        "fnt_plan_set_pipeline": (None, 1),
        "fnt_plan_set_aeq_occupancy": (None, 8),
        "fnt_plan_set_aeq_kernel": (None, 2),
        "fnt_plan_set_cdc_kernel": (None, 2),
        "fnt_plan_set_test_inject": (None, 1),
        "fnt_device_faults": (0, None),
        "fnt_plan_initial_taps": (None, None),
        "fnt_plan_set_cdc_items": (None, 0),
        "fnt_plan_set_tensor_gradient": (None, 0),
        "fnt_cdc_aeq_run_noalloc": (None, None, None),
        "fnt_session_create": (None, 1, 1 << 20, 1, None),
        "fnt_session_set_link": (None, 0, None, 5),
        "fnt_session_submit": (None, 0, None, 0, None, None),
        "fnt_session_submit_many": (None, None, 0, None, None),
        "fnt_session_cancel": (None, 1),
        "fnt_session_get_stats": (None, None),
        "fnt_session_poll": (None, 0, None, 0, None),
        "fnt_session_get_link_state": (None, 0, None),
        "fnt_session_set_link_state": (None, 0, None),
        "fnt_session_inject_failures": (None, 1),
    }
    for name, args in calls.items():
        assert getattr(L, name)(*args) == inv, name
    for name in ("fnt_plan_destroy", "fnt_batch_destroy", "fnt_session_destroy"):
        assert getattr(L, name)(None) == fnt.FNT_OK, name
    assert L.fnt_batch_kernel_count(None) == 0
    assert L.fnt_plan_aeq_kernel_for(None, 1, 1 << 20) == 0
    assert L.fnt_plan_cdc_kernel_for(None, 1) == 0
    assert L.fnt_session_pending(None) == 0
    assert fnt.last_error()                  # the last failure left its text
    decl = set(header_functions())
    covered = set(calls) | {"fnt_plan_destroy", "fnt_batch_destroy", "fnt_session_destroy", "fnt_batch_kernel_count",
                            "fnt_session_pending", "fnt_last_error", "fnt_version", "fnt_plan_desc_default",
                            "fnt_plan_aeq_kernel_for", "fnt_plan_cdc_kernel_for"}
    assert decl <= covered, decl - covered


def test_autotune_key_follows_shape_and_sources():
    """The launch-shape cache key changes with the workload's shape and with
    the library's sources (a stale entry is never reused)."""
    from types import SimpleNamespace
    from paper_2405_04253_gb300 import autotune
    plan = SimpleNamespace(desc=SimpleNamespace(n_aeq=32, aeq_segment=0, aeq_warmup=0, aeq_update_period=1))
    fr = [SimpleNamespace(n=n) for n in (4096, 70000, 9000)]
    k1 = autotune._key(plan, fr, 2)
    assert k1 == autotune._key(plan, list(reversed(fr)), 2)
    assert k1 != autotune._key(plan, fr[:2], 2)
    assert k1 != autotune._key(plan, fr, 1)
    assert k1.endswith("_src" + autotune._src_tag()) and len(autotune._src_tag()) == 12


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference launched as the driver launches N > 1 (two
    ranks, 127.0.0.1 rendezvous): rank 0 alone runs the oracle and prints one
    JSON line; the other rank exits 0 without work."""
    import json
    import socket
    import subprocess
    import sys
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-segments", "4"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"
