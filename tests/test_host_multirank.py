"""Host-side multi-rank logic on CPU (gloo, world size 2): the replicas-only bench reduces its
per-rank times with a max, and value = units of all ranks / slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 175.5][rank]
    got = bench.max_over_ranks(local_ms, world)
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == 175.5 and out[1] == 175.5


def test_max_over_ranks_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5


def test_api_fails_cleanly_without_a_device():
    # no GPU in this container: creating a context reports an argument error, never crashes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    from paper_2211_00805_gb300 import binding as gs
    h = ctypes.c_void_p()
    assert gs.lib().gs_create(ctypes.byref(h), 0, None) == gs.GS_ERR_ARG
    assert not h.value
    assert gs.lib().gs_sync(None) == gs.GS_ERR_ARG          # null context
    assert gs.lib().gs_graph_info(None, None, None, None) == gs.GS_ERR_ARG
    assert gs.lib().gs_heat_apply_noalloc(0, 0, None, None, None, 1.0, 5, None, 1, None, None) == gs.GS_ERR_ARG
