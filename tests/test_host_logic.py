"""Host-side logic that needs no GPU: ABI struct layouts of the serving API and
the multi-rank timing aggregation of bench.py (gloo, world size 2)."""
import ctypes
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _offsets_from_c(struct, fields):
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "gpe_serve.h"\nint main(void){printf("%zu' + \
        ' %zu' * len(fields) + '\\n", sizeof(%s)' % struct + ''.join(', offsetof(%s, %s)' % (struct, f) for f in fields) + \
        ');return 0;}\n'
    d = "/tmp/gpe_layout_%d_%s" % (os.getpid(), struct)
    os.makedirs(d, exist_ok=True)
    open(os.path.join(d, "c.c"), "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(d, "c.c"), "-o", os.path.join(d, "c")],
                   check=True)
    return [int(v) for v in subprocess.run([os.path.join(d, "c")], capture_output=True, text=True,
                                           check=True).stdout.split()]


@pytest.mark.parametrize("name", ["gpe_request", "gpe_result"])
def test_serving_structs_match_header(name):
    import paper_2301_08275_gb300 as gpe
    S = getattr(gpe, name)
    fields = [f for f, _ in S._fields_]
    assert _offsets_from_c(name, fields) == [ctypes.sizeof(S)] + [getattr(S, f).offset for f in fields]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(10.0 + 5.0 * rank)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_bench_reads_the_committed_traffic_file():
    """bench.py finds the DRAM bytes of every pass kind in profiles/traffic_tg512.txt
    while the kernel sources are the profiled ones (kinds contain ':')."""
    import importlib.util
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(b)
    finally:
        sys.argv = argv
    vals = {}
    for line in open(os.path.join(root, "profiles", "traffic_tg512.txt")):
        if ":" in line and not line.startswith("#"):
            k, v = line.rsplit(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != b.kernel_source_hash():
        import pytest
        pytest.skip("kernel sources changed since the traffic was profiled")
    for kind in ("x512:I-NR-F", "y512:F", "y512:I", "z512:F-KR-I"):
        t = b.read_traffic(kind, "tg512")
        assert t is not None and 1.0e9 < t < 2.2e9, (kind, t)


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one
    JSON line with the metric and unit of the GPU arm, impl=reference, a
    cpu_baseline describing the run and an e2e entry without transfers."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "TSSP grid-point updates/s vs HBM roofline" and d["unit"] == "grid-point updates/s"
    assert d["higher_is_better"] is True and d["value"] > 0 and d["warmup"] >= 3 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("3D Taylor-Green 512^3")
