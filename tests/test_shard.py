"""One bundle split over ranks by rows (paper_1601_02012_gb300.shard): the
partition, the gather of the maps and the sum of the gradients, on CPU with
two gloo ranks (127.0.0.1). Each rank's tracer here is the FP64 oracle on its
band's ray ids (the GPU path traces the same bands through rr_create_band);
the gathered map must equal the single-rank map exactly and the summed
dL/dPhi the single-rank gradient to rounding."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1601_02012_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("ny", [1, 7, 8, 9, 64, 100, 2048])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 16])
def test_bands_cover_every_row_once_in_whole_tiles(ny, world):
    bs = shard.bands(ny, world)
    assert len(bs) == world
    assert bs[0][0] == 0 and bs[-1][1] == ny
    for (a0, a1), (b0, b1) in zip(bs, bs[1:]):
        assert a1 == b0                       # contiguous, in rank order
    seen = np.zeros(ny, int)
    for y0, y1 in bs:
        assert 0 <= y0 <= y1 <= ny
        assert y0 % shard.TILE_ROWS == 0 or y0 == ny   # bands start on a tile boundary
        assert (y1 - y0) % shard.TILE_ROWS == 0 or y1 == ny
        seen[y0:y1] += 1
    assert np.all(seen == 1)
    tiles = [-(-(y1 - y0) // shard.TILE_ROWS) for y0, y1 in bs]
    assert max(tiles) - min(tiles) <= 1       # balanced to one tile
    assert shard.band_rows(ny, world - 1, world) == bs[-1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    g = synth.Grid((12, 12, 12), 24.0)
    b = synth.Bundle(10, 21, synth.deg(20), synth.deg(24), (12.0, 12.0, 0.0), 23.0)
    steps = [synth.Step(23.0, 9.0, 1.1, 0.8), synth.Step(9.0, 0.0, 0.9, 1.0)]
    phi = synth.grf_phi(12, 24.0, 17).astype(np.float64)
    rng = np.random.default_rng(3)
    dk = rng.standard_normal((b.ny, b.nx))
    return g, b, steps, phi, dk


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1601_02012_gb300 import shard as sh
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, b, steps, phi, dk = _case()
    H, d = oracle.fields(g, phi)
    y0, y1 = sh.band_rows(b.ny, rank, world)
    rids = np.arange(y0 * b.nx, y1 * b.nx)
    res = oracle.trace(b, g, H, d, steps, rids=rids) if len(rids) else None
    k = torch.from_numpy(res.kappa.reshape(y1 - y0, b.nx)) if res else torch.zeros((0, b.nx), dtype=torch.float64)
    segs = torch.tensor([float(res.nseg.sum()) if res else 0.0], dtype=torch.float64)
    k_all = sh.gather_rows(k, b.ny, rank, world)
    sh.allreduce_sum(segs, world)
    # this rank's rows of dL/dkappa through the adjoint, then the sum over ranks
    dk_band = np.zeros_like(dk)
    dk_band[y0:y1] = dk[y0:y1]
    gphi, _ = oracle.trace_adjoint(b, g, steps, dk_band)
    gt = torch.from_numpy(np.ascontiguousarray(gphi))
    sh.allreduce_sum(gt, world)
    out[rank] = (k_all.numpy(), float(segs.item()), gt.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_maps_and_sum_gradients(oracle_lib, world):
    import torch.multiprocessing as mp
    g, b, steps, phi, dk = _case()
    H, d = oracle_lib.fields(g, phi)
    whole = oracle_lib.trace(b, g, H, d, steps)
    gwhole, _ = oracle_lib.trace_adjoint(b, g, steps, dk)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        k_all, segs, gsum = res[rank]
        assert np.array_equal(k_all.ravel(), whole.kappa)
        assert segs == float(whole.nseg.sum())
        assert np.linalg.norm(gsum - gwhole) <= 1e-12 * np.linalg.norm(gwhole)
