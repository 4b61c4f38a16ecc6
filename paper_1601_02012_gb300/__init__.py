"""GB300-native line-of-sight convergence tracer (RAY-RAMSES hot path).

The computation lives in librr.so (hand-written sm_103a CUDA behind the C ABI
of include/rr.h). This package is a thin Python layer over it: ``_rr`` binds
the C entry points one to one; ``Tracer`` and ``trace_kappa`` marshal torch
tensors into them. PyTorch only provides device memory and streams.
"""
from __future__ import annotations

from . import _rr
from ._rr import (RR_AT_CENTRES, RR_AT_VERTICES, RR_NGP, RR_TRILINEAR, RRError, bundle_desc, grid_desc,
                  rr_create, rr_create_band, rr_destroy, rr_finalize, rr_footprint_bbox, rr_reset, rr_segment_count,
                  rr_status_string, rr_step_count, rr_sync_status, rr_tidal_tensor, rr_tidal_tensor_adjoint,
                  rr_trace_backward, rr_trace_step, rr_trace_step_adjoint, rr_trace_steps)

from .batch import Batch  # noqa: E402
from ._rr import rr_amr_create, rr_amr_destroy, rr_amr_sizes, rr_amr_tidal, rr_amr_trace_step  # noqa: E402
from ._rr import RR_SHEAR, rr_shear  # noqa: E402
from ._rr import RR_METHOD_A, rr_gradient_records  # noqa: E402
from ._rr import RR_GENERIC, rr_scalar_records, rr_set_kernels, rr_set_observer  # noqa: E402
from ._rr import rr_upload_box  # noqa: E402

__all__ = [
    "Batch", "AmrMesh", "source_kappa", "rr_amr_create", "rr_amr_destroy", "rr_amr_sizes", "rr_amr_tidal",
    "rr_amr_trace_step", "RR_SHEAR", "rr_shear", "RR_METHOD_A", "rr_gradient_records", "trace_method_a",
    "gradient_buffer", "RR_GENERIC", "rr_scalar_records", "rr_set_kernels", "rr_set_observer", "scalar_buffer",
    "trace_tiles", "rr_upload_box",
    "Tracer", "pipeline_steps", "box_record_buffer", "trace_kappa", "trace_shear", "record_buffer", "grad_buffer", "RRError", "rr_create", "rr_destroy", "rr_reset",
    "rr_tidal_tensor", "rr_footprint_bbox", "rr_trace_step", "rr_finalize", "rr_sync_status",
    "rr_segment_count", "rr_status_string", "rr_step_count", "rr_trace_step_adjoint", "rr_tidal_tensor_adjoint",
    "rr_trace_backward", "rr_trace_steps", "TraceKappa", "RR_NGP", "RR_TRILINEAR", "RR_AT_VERTICES", "RR_AT_CENTRES",
]


def scalar_buffer(grid, device="cuda"):
    """Zeroed device buffer for n0*n1*n2 scalar-pair records (generic form)."""
    import torch
    n = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
    return torch.zeros((n, 2), dtype=torch.float32, device=device)


def gradient_buffer(grid, device="cuda"):
    """Uninitialised device buffer for n0*n1*n2 gradient records of 4 floats
    (Method A)."""
    import torch
    n = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
    return torch.empty((n, 4), dtype=torch.float32, device=device)


def record_buffer(grid, device="cuda"):
    """Uninitialised device buffer for n0*n1*n2 records of 8 floats."""
    import torch
    n = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
    return torch.empty((n, 8), dtype=torch.float32, device=device)


def box_record_buffer(bbox, device="cuda"):
    """Uninitialised device buffer for the box-local records of a box
    (rr_tidal_tensor_box): 8 floats per point of the box."""
    import torch
    n = (int(bbox[1]) - int(bbox[0])) * (int(bbox[3]) - int(bbox[2])) * (int(bbox[5]) - int(bbox[4]))
    return torch.empty((n, 8), dtype=torch.float32, device=device)


def grad_buffer(grid, device="cuda"):
    """Uninitialised device buffer for n0*n1*n2 gradient records of 64 bytes
    (16 floats' room: the 8 record channels as FP64 sums)."""
    import torch
    n = int(grid.n[0]) * int(grid.n[1]) * int(grid.n[2])
    return torch.empty((n, 16), dtype=torch.float32, device=device)


class Tracer:
    """One ray bundle's device state (an rr_ctx) plus the calls that advance it.

    bundle: object with nx, ny, fov_x, fov_y (radians), obs (3), chi_s, interp
    (0 NGP / 1 trilinear) and periodic attributes. fp64_dda: the plain FP64
    walk; plain_sums: the FP32 walk without compensated sums (for comparison);
    moments: accumulate the source-redshift moments of Eq. (Isources) (see
    ``moments()`` and ``source_kappa``); shear: also accumulate the shear
    (gamma1, gamma2) of Eqs. gamma1, gamma2 in the same walk (see ``shear()``);
    method_a: kappa by Method A (Eq. kappa2) from gradient records
    (``tidal`` then writes those, 4 floats per point); generic: two generic
    integrals int K_c Q_c dchi from scalar-pair records (see ``scalars``,
    ``set_kernels``).
    """

    def __init__(self, bundle, fp64_dda: bool = False, plain_sums: bool = False, moments: bool = False,
                 shear: bool = False, method_a: bool = False, generic: bool = False, rows=None):
        _rr.load()
        self.bundle = bundle
        self.method_a = bool(method_a)
        self.generic = bool(generic)
        self.desc = bundle_desc(bundle, fp64_dda=fp64_dda, plain_sums=plain_sums, moments=moments, shear=shear,
                                method_a=method_a, generic=generic)
        # rows (y0, y1): this tracer's rays are that band of the bundle (rr_create_band)
        self.rows = (0, int(bundle.ny)) if rows is None else (int(rows[0]), int(rows[1]))
        self.ctx = rr_create(self.desc) if rows is None else rr_create_band(self.desc, *self.rows)
        self.where = RR_AT_VERTICES if int(self.desc.interp) == RR_TRILINEAR else RR_AT_CENTRES

    def close(self):
        if getattr(self, "ctx", None) is not None:
            rr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        rr_reset(self.ctx, stream)

    def tidal(self, grid, phi, rec, delta=None, bbox=None, stream=None):
        """The records this context traces, into ``rec``, at vertices
        (trilinear) or centres (NGP): rr_tidal_tensor, or rr_gradient_records
        for Method A."""
        if self.method_a:
            _rr.rr_gradient_records(grid_desc(grid), phi, delta, rec, self.where, bbox, stream)
        else:
            rr_tidal_tensor(grid_desc(grid), phi, delta, rec, self.where, bbox, stream)
        return rec

    def record_buffer(self, grid, device="cuda"):
        """An uninitialised record buffer of the kind this context traces."""
        if self.generic:
            return scalar_buffer(grid, device)
        return gradient_buffer(grid, device) if self.method_a else record_buffer(grid, device)

    def scalars(self, grid, field, rec, channel=0, field_prev=None, inv_dt=1.0, bbox=None, stream=None):
        """rr_scalar_records: channel ``channel`` of the scalar-pair records."""
        _rr.rr_scalar_records(grid_desc(grid), field, field_prev, inv_dt, channel, rec, self.where, bbox, stream)
        return rec

    def set_kernels(self, kernels):
        """(k0, k1, k2) per channel: K_c(chi) = k0 + k1 chi + k2 chi^2."""
        _rr.rr_set_kernels(self.ctx, kernels)

    def set_observer(self, obs):
        """Move the observer for the following steps (box tiling, Sec. 2.2)."""
        _rr.rr_set_observer(self.ctx, obs)
        self.desc.obs[0], self.desc.obs[1], self.desc.obs[2] = (float(x) for x in obs)

    def footprint(self, grid, chi_a, chi_b, pad=0):
        """rr_footprint_bbox of the step, widened by ``pad`` points per side
        (an axis it would cover whole becomes [0, n)); pad=1 gives the boxes
        rr_trace_steps takes with box-local records."""
        bb = list(rr_footprint_bbox(self.desc, grid_desc(grid), chi_a, chi_b))
        for a in range(3):
            n = int(grid.n[a])
            if bb[2 * a + 1] - bb[2 * a] + 2 * pad >= n:
                bb[2 * a], bb[2 * a + 1] = 0, n
            else:
                bb[2 * a] -= pad
                bb[2 * a + 1] += pad
        return tuple(bb)

    def step(self, grid, rec, chi_a, chi_b, scale=1.0, a=1.0, stream=None):
        rr_trace_step(self.ctx, grid_desc(grid), rec, chi_a, chi_b, scale, a, stream)

    def steps(self, grid, recs, steps, boxes=None, stream=None):
        """rr_trace_steps: the given steps (objects with chi_a, chi_b, scale,
        a) in order, step i reading recs[i] (whole-grid records, or, with
        ``boxes``, the box-local records of box i); the default form traces up
        to 16 of them per launch."""
        _rr.rr_trace_steps(self.ctx, grid_desc(grid), list(recs), [st.chi_a for st in steps],
                           [st.chi_b for st in steps], [st.scale for st in steps], [st.a for st in steps],
                           boxes, stream)

    def tidal_box(self, grid, phi, rec, bbox, delta=None, stream=None):
        """rr_tidal_tensor_box: the records of the points of ``bbox`` only,
        box-local, into ``rec`` (box_record_buffer)."""
        _rr.rr_tidal_tensor_box(grid_desc(grid), phi, delta, rec, self.where, bbox, stream)
        return rec

    def finalize(self, kappa=None, kborn=None, stream=None):
        """FP64 maps [ny, nx] on the device (rayid order, x fastest)."""
        import torch
        ny, nx = self.rows[1] - self.rows[0], int(self.desc.nx)
        if kappa is None:
            kappa = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        if kborn is None:
            kborn = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        rr_finalize(self.ctx, kappa, kborn, stream)
        return kappa, kborn

    def segments(self, per_ray=None, stream=None) -> int:
        return rr_segment_count(self.ctx, per_ray, stream)

    def moments(self, out=None, stream=None):
        """Snapshot of the moments so far: FP64 [4, ny, nx] on the device, rows
        A_kappa, B_kappa, A_born, B_born (contexts created with moments=True)."""
        import torch
        ny, nx = self.rows[1] - self.rows[0], int(self.desc.nx)
        if out is None:
            out = torch.empty((4, ny, nx), dtype=torch.float64, device="cuda")
        _rr.rr_moments(self.ctx, out, stream)
        return out

    def shear(self, gamma1=None, gamma2=None, stream=None):
        """The shear maps so far: FP64 (gamma1, gamma2), each [ny, nx] on the
        device (contexts created with shear=True)."""
        import torch
        ny, nx = self.rows[1] - self.rows[0], int(self.desc.nx)
        if gamma1 is None:
            gamma1 = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        if gamma2 is None:
            gamma2 = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        _rr.rr_shear(self.ctx, gamma1, gamma2, stream)
        return gamma1, gamma2

    def trace_streamed(self, grid, phi_host, steps, rec, bufs, stream, copy_stream, bboxes=None, delta_host=None,
                       delta_bufs=None, group=1, box_recs=None, rec_stream=None):
        """The steps of a pass with the potential streamed from host memory.

        phi_host: page-locked host tensor of n0*n1*n2 floats; bufs: two device
        arrays of the same size; steps: objects with chi_a, chi_b, scale, a.
        For each step rr_upload_box copies the step's footprint (plus the
        stencil reach) into one of the two buffers on ``copy_stream`` while the
        step before computes from the other one; ``stream`` waits for each
        copy before the step's records, and a copy into a buffer waits until
        the records made from it two steps earlier are done. Only the cells a
        step reads are moved, so the maps equal those of the same steps on the
        whole field. delta_host / delta_bufs: the same for a given density
        contrast. The host arrays must stay unchanged until ``stream`` has
        passed the last step. group > 1: each step's records go into its own
        box-local buffer box_recs[i] over bboxes[i] (footprints widened by one
        point: footprint(pad=1)), and every ``group`` steps are traced by one
        rr_trace_steps call; with ``rec_stream`` (a higher-priority stream)
        those records are computed there, beside the previous group's trace,
        and each group's trace waits for its own. Returns the bytes copied."""
        import torch
        if self.generic:
            raise ValueError("trace_streamed: the generic form takes its fields through scalars()")
        if group > 1 and (box_recs is None or bboxes is None):
            raise ValueError("trace_streamed: group > 1 takes box_recs and their (padded) bboxes")
        g = grid_desc(grid)
        if bboxes is None:
            bboxes = [self.footprint(grid, st.chi_a, st.chi_b) for st in steps]
        # the buffers may still be read by work already queued on `stream`
        # (a previous pass): the first copies wait for it
        queued = torch.cuda.Event()
        queued.record(stream)
        copy_stream.wait_event(queued)
        rs = rec_stream if (group > 1 and rec_stream is not None) else stream
        if rs is not stream:
            rs.wait_event(queued)
        released = [None, None]
        total = 0
        for i, st in enumerate(steps):
            slot = i % 2
            if released[slot] is not None:
                copy_stream.wait_event(released[slot])
            total += rr_upload_box(g, phi_host, bufs[slot], bboxes[i], copy_stream)
            delta = None
            if delta_host is not None:
                total += rr_upload_box(g, delta_host, delta_bufs[slot], bboxes[i], copy_stream)
                delta = delta_bufs[slot]
            copied = torch.cuda.Event()
            copied.record(copy_stream)
            rs.wait_event(copied)
            if group > 1:
                self.tidal_box(grid, bufs[slot], box_recs[i], bboxes[i], delta=delta, stream=rs)
            else:
                self.tidal(grid, bufs[slot], rec, delta=delta, bbox=bboxes[i], stream=rs)
            done = torch.cuda.Event()
            done.record(rs)
            released[slot] = done
            if group <= 1:
                self.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream)
            elif (i + 1) % group == 0 or i == len(steps) - 1:
                k0 = i - i % group
                if rs is not stream:
                    stream.wait_event(done)   # the group's records (rs runs them in order)
                self.steps(grid, box_recs[k0:i + 1], steps[k0:i + 1], boxes=bboxes[k0:i + 1], stream=stream)
        return total

    def amr_steps(self, mesh, leaf_recs, steps, stream=None):
        """rr_amr_trace_steps: the given steps over ``mesh`` in order, step i
        reading leaf_recs[i]; the default form traces up to 16 per launch."""
        _rr.rr_amr_trace_steps(self.ctx, mesh.handle, list(leaf_recs), [st.chi_a for st in steps],
                               [st.chi_b for st in steps], [st.scale for st in steps], [st.a for st in steps],
                               stream)

    def amr_step(self, mesh, leaf_rec, chi_a, chi_b, scale=1.0, a=1.0, stream=None):
        """One step over an adaptive mesh (``AmrMesh``) from its leaf records."""
        rr_amr_trace_step(self.ctx, mesh.handle, leaf_rec, chi_a, chi_b, scale, a, stream)

    def backward(self, grid, dkappa, dkborn=None, grad_rec=None, dphi=None, ddelta=None, stream=None):
        """dL/dPhi (and dL/ddelta if ``ddelta`` is given: delta was an input)
        for all logged steps, through rr_trace_backward."""
        import torch
        n = tuple(int(x) for x in grid.n)
        dev = (dkappa if dkappa is not None else dkborn).device
        if grad_rec is None:
            grad_rec = grad_buffer(grid, device=dev)
        if dphi is None:
            dphi = torch.zeros(n, dtype=torch.float32, device=dev)
        rr_trace_backward(self.ctx, dkappa.contiguous() if dkappa is not None else None,
                          dkborn.contiguous() if dkborn is not None else None, grad_rec, dphi, ddelta, stream)
        return dphi


def source_kappa(m_end, m_k, chi_k, stream=None):
    """kappa and Born kappa [ny, nx] for sources at chi_k from two moment
    snapshots (``Tracer.moments``): m_end after the last step, m_k after the
    steps down to chi_k (None when chi_k is the bundle's chi_s)."""
    import torch
    ny, nx = int(m_end.shape[1]), int(m_end.shape[2])
    k = torch.empty((ny, nx), dtype=torch.float64, device=m_end.device)
    kb = torch.empty_like(k)
    _rr.rr_source_kappa(m_end, m_k, ny * nx, chi_k, k, kb, stream)
    return k, kb


class AmrMesh:
    """An adaptive mesh's device plan (an rr_amr).

    n, lmax, box, omega_m: coarse cells per side, finest level, extent, Omega_m.
    octs[l] (l = 1..lmax): [m_l, 3] integer coordinates of the level-(l-1)
    cells refined into level-l octs. Cells are numbered level 0 row-major,
    then per level oct after oct (in the given order) x 8 children.
    """

    def __init__(self, n, lmax, box, octs, omega_m=0.3):
        _rr.load()
        d = _rr.rr_amr_desc()
        d.n, d.lmax, d.box, d.omega_m = int(n), int(lmax), float(box), float(omega_m)
        self.desc = d
        self.handle = rr_amr_create(d, octs)
        self.ncells, self.nleaves, self.nverts = rr_amr_sizes(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            rr_amr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def record_buffer(self, where=RR_AT_VERTICES, device="cuda"):
        """Uninitialised leaf records: 64 floats per leaf at vertices, 8 at centres."""
        import torch
        per = 64 if where == RR_AT_VERTICES else 8
        return torch.empty((self.nleaves, per), dtype=torch.float32, device=device)

    def tidal(self, phi, leaf_rec, where=RR_AT_VERTICES, cell_tidal=None, bbox=None, stream=None):
        """rr_amr_tidal: phi (float32 [ncells], cell order) -> leaf records
        (of the leaves in ``bbox``, a coarse-cell box, or of all)."""
        rr_amr_tidal(self.handle, phi, where, leaf_rec, cell_tidal, bbox, stream)
        return leaf_rec

    def gradient(self, phi, leaf_rec, where=RR_AT_VERTICES, cell_grad=None, bbox=None, stream=None):
        """rr_amr_gradient: the Method A records ({grad Phi, 0}, {0, 0, delta,
        0} in the layout of the tidal records) of the leaves in ``bbox`` or of all."""
        _rr.rr_amr_gradient(self.handle, phi, where, leaf_rec, cell_grad, bbox, stream)
        return leaf_rec

    def scalars(self, field0, leaf_rec, where=RR_AT_VERTICES, prev0=None, inv_dt0=1.0, field1=None, prev1=None,
                inv_dt1=1.0, cell_buf=None, bbox=None, stream=None):
        """rr_amr_scalars: the records of the generic integrals, channel c the
        field (cell order) or (field - prev) * inv_dt; field1 None: zero."""
        _rr.rr_amr_scalars(self.handle, field0, prev0, inv_dt0, field1, prev1, inv_dt1, where, leaf_rec, cell_buf,
                           bbox, stream)
        return leaf_rec

    def coarse_grid(self):
        """rr_grid_desc of the coarse grid (for rr_footprint_bbox)."""
        d = _rr.rr_grid_desc()
        for i in range(3):
            d.n[i] = int(self.desc.n)
        d.box, d.omega_m = float(self.desc.box), float(self.desc.omega_m)
        return d

    def footprint(self, tracer, chi_a, chi_b):
        """Coarse-cell box of the leaves a step of ``tracer``'s bundle can read."""
        return rr_footprint_bbox(tracer.desc, self.coarse_grid(), chi_a, chi_b)


def pipeline_steps(n, records, trace, stream, side=None, nbuf=1, timing=None):
    """Issue the n steps of a pass: ``records(i, b, s)`` computes step i's
    records into buffer b on stream s, ``trace(i, b, s)`` traces step i from
    buffer b on s. With one buffer (or no side stream) both run in order on
    ``stream``. With two buffers and a side stream the records of step i + 1
    are computed on ``side`` while step i is traced on ``stream``: step i's
    trace waits for its records, and the records written into a buffer wait
    for the trace that last read it (each step reads only its own footprint,
    which its records cover). The side stream starts after the work already
    on ``stream``; everything ends on ``stream``. Give ``side`` a higher
    priority than ``stream`` (torch.cuda.Stream(priority=-1)): the records'
    few blocks are then placed as soon as trace blocks retire, and are ready
    before the trace they feed. ``timing``: two lists of n
    (start, end) CUDA event pairs, recorded around each step's records and
    its trace."""
    import torch
    rec_ev, tr_ev = timing if timing is not None else (None, None)

    def rec(i, b, s):
        if rec_ev is not None:
            rec_ev[i][0].record(s)
        records(i, b, s)
        if rec_ev is not None:
            rec_ev[i][1].record(s)

    def tra(i, b, s):
        if tr_ev is not None:
            tr_ev[i][0].record(s)
        trace(i, b, s)
        if tr_ev is not None:
            tr_ev[i][1].record(s)

    if side is None or nbuf < 2:
        for i in range(n):
            rec(i, 0, stream)
            tra(i, 0, stream)
        return
    start = torch.cuda.Event()
    start.record(stream)
    side.wait_event(start)
    ready = [torch.cuda.Event() for _ in range(n)]
    used = [torch.cuda.Event() for _ in range(n)]
    if n > 0:
        rec(0, 0, side)
        ready[0].record(side)
    for i in range(n):
        if i + 1 < n:
            if i >= 1:
                side.wait_event(used[i - 1])   # buffer (i + 1) % 2 was last read by step i - 1
            rec(i + 1, (i + 1) % 2, side)
            ready[i + 1].record(side)
        stream.wait_event(ready[i])
        tra(i, i % 2, stream)
        used[i].record(stream)


def trace_kappa(phi, grid, bundle, steps, delta=None, fp64_dda=False, footprint=True, stream=None, group=16):
    """Trace a bundle through a sequence of steps on one potential.

    phi: device float32 tensor n0 x n1 x n2 (Phi/c^2 at cell centres).
    steps: objects with chi_a, chi_b, scale, a (the step's field is scale * Phi).
    For each step the records are recomputed (restricted to the step's
    footprint when ``footprint``) and the bundle is advanced; returns the FP64
    (kappa, kappa_born) maps and the number of cell segments. For a periodic
    trilinear bundle in the FP32 walk whose steps' footprints (widened by a
    point) are smaller than the grid, each step's records are computed over
    its footprint box only (box-local) and ``group`` steps are traced per
    launch (rr_trace_steps; the same maps bit for bit); group=1: one
    rr_trace_step per step on whole-grid records.
    """
    tr = Tracer(bundle, fp64_dda=fp64_dda)
    try:
        boxes = None
        if group > 1 and footprint and not fp64_dda and int(bundle.interp) == RR_TRILINEAR and \
                (int(tr.desc.flags) & _rr.RR_PERIODIC):
            boxes = [tr.footprint(grid, st.chi_a, st.chi_b, pad=1) for st in steps]
            if any(bb[2 * a + 1] - bb[2 * a] >= int(grid.n[a]) for bb in boxes for a in range(3)):
                boxes = None
        if boxes is not None:
            recs = [box_record_buffer(bb, device=phi.device) for bb in boxes]
            for i in range(0, len(steps), group):
                for k in range(i, min(i + group, len(steps))):
                    tr.tidal_box(grid, phi, recs[k], boxes[k], delta=delta, stream=stream)
                tr.steps(grid, recs[i:i + group], steps[i:i + group], boxes=boxes[i:i + group], stream=stream)
        else:
            rec = record_buffer(grid, device=phi.device)
            for st in steps:
                bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
                tr.tidal(grid, phi, rec, delta=delta, bbox=bbox, stream=stream)
                tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream=stream)
        k, kb = tr.finalize(stream=stream)
        return k, kb, tr.segments()
    finally:
        tr.close()


def trace_method_a(phi, grid, bundle, steps, delta=None, footprint=True, stream=None):
    """As ``trace_kappa``, by Method A (Eq. kappa2): the records are the
    gradient records, and the returned kappa holds the density term, the
    integral of (1 - 2 chi/chi_s) n.grad(Phi) and the steps' surface terms;
    kappa_born is the density term alone."""
    tr = Tracer(bundle, method_a=True)
    try:
        rec = tr.record_buffer(grid, device=phi.device)
        for st in steps:
            bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
            tr.tidal(grid, phi, rec, delta=delta, bbox=bbox, stream=stream)
            tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream=stream)
        k, kb = tr.finalize(stream=stream)
        return k, kb, tr.segments()
    finally:
        tr.close()


def trace_tiles(tiles, bundle, steps, footprint=True, stream=None):
    """Trace one bundle through a tile of boxes (Sec. 2.2): ``tiles`` is a list
    of (phi, grid, obs) with the observer's position relative to each box's
    origin; each box is traced over all ``steps`` from its own observer, and
    without wrap (the bundle's periodic flag is ignored) a ray contributes only
    while it is inside that box. Returns the FP64 (kappa, kappa_born) maps of
    the whole tile and the number of cell segments."""
    import copy
    b = copy.copy(bundle)
    b.periodic = False
    tr = Tracer(b)
    try:
        for phi, grid, obs in tiles:
            rec = record_buffer(grid, device=phi.device)
            tr.set_observer(obs)
            for st in steps:
                bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
                tr.tidal(grid, phi, rec, bbox=bbox, stream=stream)
                tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream=stream)
        k, kb = tr.finalize(stream=stream)
        return k, kb, tr.segments()
    finally:
        tr.close()


def trace_shear(phi, grid, bundle, steps, delta=None, footprint=True, stream=None):
    """As ``trace_kappa``, with the shear of Eqs. gamma1, gamma2 accumulated in
    the same walk: returns the FP64 maps (kappa, kappa_born, gamma1, gamma2),
    each [ny, nx], and the number of cell segments."""
    tr = Tracer(bundle, shear=True)
    try:
        rec = record_buffer(grid, device=phi.device)
        for st in steps:
            bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
            tr.tidal(grid, phi, rec, delta=delta, bbox=bbox, stream=stream)
            tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a, stream=stream)
        k, kb = tr.finalize(stream=stream)
        g1, g2 = tr.shear(stream=stream)
        return k, kb, g1, g2, tr.segments()
    finally:
        tr.close()


def _make_autograd():
    import torch

    class TraceKappa(torch.autograd.Function):
        """(kappa, kappa_born) = trace(phi) as a differentiable torch op.

        forward: rr_tidal_tensor + rr_trace_step per step + rr_finalize;
        backward: rr_trace_backward (the hand-written adjoint), giving dL/dPhi
        for the FP32 potential. The maps are FP64, shaped [ny, nx].
        """

        @staticmethod
        def forward(ctx, phi, grid, bundle, steps, footprint=True):
            tr = Tracer(bundle)
            rec = record_buffer(grid, device=phi.device)
            for st in steps:
                bbox = tr.footprint(grid, st.chi_a, st.chi_b) if footprint else None
                tr.tidal(grid, phi.detach().contiguous(), rec, bbox=bbox)
                tr.step(grid, rec, st.chi_a, st.chi_b, st.scale, st.a)
            k, kb = tr.finalize()
            ctx.tracer = tr
            ctx.grid = grid
            return k, kb

        @staticmethod
        def backward(ctx, gk, gb):
            tr = ctx.tracer
            dphi = tr.backward(ctx.grid, gk.contiguous() if gk is not None else None,
                               gb.contiguous() if gb is not None else None)
            tr.close()
            return dphi, None, None, None, None

    return TraceKappa


class _Lazy:
    _fn = None

    def __getattr__(self, name):
        if _Lazy._fn is None:
            _Lazy._fn = _make_autograd()
        return getattr(_Lazy._fn, name)


#: torch.autograd.Function: TraceKappa.apply(phi, grid, bundle, steps) -> (kappa, kappa_born)
TraceKappa = _Lazy()
