"""The multi-GPU form of the bench is independent replicas (the path is not
sharded): each rank times its own problem and the job's time is the largest
over the ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    ws, r, _ = bench.dist_setup()
    got = bench.max_over_ranks(10.0 + 3.0 * rank, dist)
    ref = bench.run_reference(None, ws, r) if r != 0 else 'rank0'   # ranks > 0 do no reference work
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, ws, got, ref))


def test_two_gloo_ranks_take_the_max_time():
    torch = pytest.importorskip('torch')
    import torch.multiprocessing as mp
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2, 2]
    assert all(r[2] == 13.0 for r in res)          # the slower rank's time on every rank
    assert res[1][3] is None                       # rank 1 prints nothing for the reference arm


def test_single_process_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.5) == 4.5


def test_profiled_traffic_only_for_unchanged_kernel(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from the committed ncu summary only
    while the tuned configuration and the kernel's sources are the ones the
    capture was taken with."""
    import bench
    h = bench.sources_sha256(bench.TRAFFIC_SOURCES)
    summ = tmp_path / 'summary.md'
    summ.write_text('# summary\n\ntraffic_record: cfg=7,1,32 dram_bytes_per_launch=123456 sources_sha256=%s\n' % h)
    monkeypatch.setattr(bench, 'TRAFFIC_SUMMARY', str(summ))
    assert bench.profiled_traffic((7, 1, 32)) == (123456, str(summ))
    v, why = bench.profiled_traffic((3, 1, 32))
    assert v is None and 'configuration' in why
    summ.write_text('traffic_record: cfg=7,1,32 dram_bytes_per_launch=123456 sources_sha256=%s\n' % ('0' * 64))
    v, why = bench.profiled_traffic((7, 1, 32))
    assert v is None and 'changed' in why
    monkeypatch.setattr(bench, 'TRAFFIC_SUMMARY', str(tmp_path / 'absent.md'))
    assert bench.profiled_traffic((7, 1, 32))[0] is None
