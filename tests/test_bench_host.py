"""Host-side logic of bench.py (no GPU): the per-stage byte accounting and the
rule that reports ncu DRAM traffic only for the kernel sources it was taken on."""
import os

import pytest

import bench


def test_stage_bytes_add_up_to_the_call():
    """At Nq = 20 on 180 points along x: the per-stage algorithmic bytes match
    the names of the library's stages, the contraction moves the half
    spectrum in and out once, and the whole call moves more than the
    396 B/pt floor (the y stage is three passes over the spectrum)."""
    from paper_0812_0244_gb300 import vdwnl
    sb = bench.stage_bytes_per_point(20, 180)
    assert tuple(sb) == vdwnl.VdwNL.STAGES
    h = 91 / 180
    assert sb["pointwise"] == pytest.approx(117)
    assert sb["contract"] == pytest.approx(2 * 20 * 8 * h + 4 * h)
    assert sb["pencils_fwd"] == sb["pencils_inv"] == pytest.approx(2 * 20 * 8 * h)
    assert sum(sb.values()) == pytest.approx(117 + 160.9 + 3 * 161.8 + 2 + 160.9 + 109 + 28.1 + 16.2 + 12.0, abs=0.2)
    assert bench.b_alg(20) == 396 < sum(sb.values())


def test_contraction_flops_and_fp32_peak():
    """Nq = 20: 210 pair evaluations of 3 FMA, 4 FMA per off-diagonal and 2 per
    diagonal pair, 2 FMA per field of energy, 2 products per field of
    scaling: 2980 flops per half-spectrum point; the FP32 peak at 2070 MHz is
    152 x 128 x 2 x 2.07e9 = 80.5 TFLOP/s."""
    assert bench.contract_flops_per_point(20, 180) == pytest.approx(2980 * 91 / 180)
    assert bench.fp32_peak_tflops(2070) == pytest.approx(80.55, abs=0.01)


def test_traffic_reported_only_for_matching_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_0812_0244_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "pipeline.cu").write_text("kernel one")
    (csrc / "learned.cu").write_text("other kernels")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha1()
    (tmp_path / "profiles" / "dram_traffic_dwnt_180x180x72_nq20.txt").write_text(
        "# comment\nsource_sha1 %s\ncontract 123456\n" % sha)
    assert bench.captured_traffic("contract") == 123456
    assert bench.captured_traffic("usum") is None  # not captured
    (csrc / "learned.cu").write_text("other kernels, changed")  # not a plain-path source
    assert bench.source_sha1() == sha
    (csrc / "pipeline.cu").write_text("kernel two")               # sources changed since the capture
    assert bench.source_sha1() != sha
    assert bench.captured_traffic("contract") is None


def test_committed_traffic_file_names_its_sources():
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "dram_traffic_dwnt_180x180x72_nq20.txt")
    keys = [line.split()[0] for line in open(path) if line.strip() and not line.startswith("#")]
    assert keys[0] == "source_sha1" and "contract" in keys


def _replica_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.slowest_rank(1.0 + rank, world)   # rank r took 1 + r ms
        dist.barrier()
        out[rank] = ms
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    """The N > 1 path of bench.py (replicas, one cell per rank): every rank
    ends with the slowest rank's time, so value = world x points / max time.
    Two gloo ranks on the CPU."""
    torch = pytest.importorskip("torch")
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 2.0, 1: 2.0}
    assert bench.slowest_rank(3.5, 1) == 3.5
