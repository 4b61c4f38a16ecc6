"""One bundle traced on several GPUs, one process per GPU.

Rays are independent: the paper exchanges rays between processes only because
it splits the simulation volume among them (Secs. 2.3-2.5). Here every rank
holds the whole potential and traces a band of the bundle's pixel rows
(``rr_create_band``), made of whole ray tiles of the trace kernel, with no
exchange while tracing. The forward's one collective gathers the maps: the
whole map is the bands' maps concatenated in row order (Eq. rayid is row
major). The adjoint's one collective sums dL/dPhi over the ranks: each rank
back-propagates its own rows of dL/dkappa through its own band, and the
gradient of the whole bundle is the sum of the bands' gradients.

The collectives are torch.distributed calls (NCCL on GPUs, gloo on CPUs);
everything between them runs in the library's kernels.
"""
from __future__ import annotations

#: rows of one block of the trace kernel's default ray tile (2 x 2 warps of
#: 8 x 4 pixels): bands made of whole tiles launch the same blocks as the
#: whole bundle does
TILE_ROWS = 8


def bands(ny: int, world: int, tile_rows: int = TILE_ROWS) -> list:
    """The row bands [y0, y1) of ``world`` ranks over ``ny`` rows: whole tiles
    of ``tile_rows`` rows, as even as possible, lower ranks taking the spare
    tiles; a rank may get an empty band when there are fewer tiles than ranks."""
    if ny < 0 or world < 1 or tile_rows < 1:
        raise ValueError("bands: ny >= 0, world >= 1, tile_rows >= 1")
    ntiles = -(-ny // tile_rows)
    base, extra = divmod(ntiles, world)
    out = []
    t0 = 0
    for r in range(world):
        t1 = t0 + base + (1 if r < extra else 0)
        out.append((min(t0 * tile_rows, ny), min(t1 * tile_rows, ny)))
        t0 = t1
    return out


def band_rows(ny: int, rank: int, world: int, tile_rows: int = TILE_ROWS) -> tuple:
    """Rank ``rank``'s band [y0, y1) of ``bands``."""
    return bands(ny, world, tile_rows)[rank]


def gather_rows(local, ny: int, rank: int, world: int, group=None, tile_rows: int = TILE_ROWS):
    """The whole [ny, nx] map on every rank from each rank's band ``local``
    ([y1 - y0, nx]): an all-gather of the bands (padded to the largest),
    concatenated in row order."""
    import torch
    import torch.distributed as dist
    bs = bands(ny, world, tile_rows)
    y0, y1 = bs[rank]
    if tuple(local.shape[:1]) != (y1 - y0,):
        raise ValueError(f"gather_rows: rank {rank} holds {local.shape[0]} rows, its band has {y1 - y0}")
    if world == 1:
        return local
    rows = max(b1 - b0 for b0, b1 in bs)
    pad = torch.zeros((rows,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: y1 - y0] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[: b1 - b0] for p, (b0, b1) in zip(parts, bs)], dim=0)


def allreduce_sum(t, world: int, group=None):
    """Sum of ``t`` over the ranks, in place (the adjoint's one collective)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def trace_kappa_sharded(phi, grid, bundle, steps, rank: int, world: int, group=None, footprint: bool = True,
                        stream=None):
    """``trace_kappa`` with the bundle's rows split over the ranks: every rank
    passes the same potential and steps, traces its band and returns the
    whole (kappa, kappa_born) maps and the whole bundle's segment count."""
    import torch
    from . import Tracer, record_buffer
    y0, y1 = band_rows(int(bundle.ny), rank, world)
    nx = int(bundle.nx)
    segs = 0
    if y1 > y0:
        tr = Tracer(bundle, rows=(y0, y1))
        try:
            rec = record_buffer(grid, device=phi.device)
            for st in steps:
                bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
                tr.tidal(grid, phi, rec, bbox=bbox, stream=stream)
                tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream=stream)
            k, kb = tr.finalize(stream=stream)
            segs = tr.segments()
        finally:
            tr.close()
    else:
        k = torch.empty((0, nx), dtype=torch.float64, device=phi.device)
        kb = torch.empty_like(k)
    n = torch.tensor([segs], dtype=torch.float64, device=phi.device)
    allreduce_sum(n, world, group)
    return (gather_rows(k, int(bundle.ny), rank, world, group), gather_rows(kb, int(bundle.ny), rank, world, group),
            int(n.item()))


def _make_autograd():
    import torch

    class ShardedTraceKappa(torch.autograd.Function):
        """(kappa, kappa_born) = trace(phi) with the rows split over the ranks.

        Every rank passes the same phi and gets the whole maps; backward takes
        this rank's rows of dL/dkappa through rr_trace_backward of its band and
        sums dL/dPhi over the ranks, so every rank gets the whole gradient of a
        loss that each rank evaluates on the whole maps."""

        @staticmethod
        def forward(ctx, phi, grid, bundle, steps, rank, world, group=None, footprint=True):
            from . import Tracer, record_buffer
            y0, y1 = band_rows(int(bundle.ny), rank, world)
            tr = None
            if y1 > y0:
                tr = Tracer(bundle, rows=(y0, y1))
                rec = record_buffer(grid, device=phi.device)
                for st in steps:
                    bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
                    tr.tidal(grid, phi.detach().contiguous(), rec, bbox=bbox)
                    tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
                k, kb = tr.finalize()
            else:
                k = torch.empty((0, int(bundle.nx)), dtype=torch.float64, device=phi.device)
                kb = torch.empty_like(k)
            ctx.tracer, ctx.grid, ctx.rows, ctx.world, ctx.group = tr, grid, (y0, y1), world, group
            ctx.shape = tuple(phi.shape)
            ny = int(bundle.ny)
            return gather_rows(k, ny, rank, world, group), gather_rows(kb, ny, rank, world, group)

        @staticmethod
        def backward(ctx, gk, gb):
            y0, y1 = ctx.rows
            tr = ctx.tracer
            if tr is not None:
                dphi = tr.backward(ctx.grid, gk[y0:y1].contiguous() if gk is not None else None,
                                   gb[y0:y1].contiguous() if gb is not None else None)
                tr.close()
            else:
                dev = (gk if gk is not None else gb).device
                dphi = torch.zeros(ctx.shape, dtype=torch.float32, device=dev)
            allreduce_sum(dphi, ctx.world, ctx.group)
            return dphi, None, None, None, None, None, None, None

    return ShardedTraceKappa


class _Lazy:
    _fn = None

    def __getattr__(self, name):
        if _Lazy._fn is None:
            _Lazy._fn = _make_autograd()
        return getattr(_Lazy._fn, name)


#: torch.autograd.Function: ShardedTraceKappa.apply(phi, grid, bundle, steps, rank, world[, group])
ShardedTraceKappa = _Lazy()
