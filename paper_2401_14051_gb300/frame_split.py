"""One frame's shading split across processes, one process per GPU.

The paper evaluates many network instances in parallel over independent shading points
(Sec. III.C.2, input batching).  Here each rank shades one contiguous range of a frame's
shading points and rank 0 assembles the image:

* replicated on every rank: the volume (uploaded by each), its pyramid and transmittance
  (each rank builds its own), the weights and the phase table;
* per rank: ``Context.render_frame_part`` finds the frame's hits, lists them in pixel order
  (the same list on every rank) and shades range ``rank`` of ``world`` of it (equal
  contiguous ranges, ``nis.part_range``);
* the one exchange: ``gather_parts`` sends each range's radiance and pixel indices to the
  destination rank, which scatters them into the image with ``Context.scatter_part``.

Every step on the data path runs in the library's kernels; this module only moves buffers
between ranks (``torch.distributed``, NCCL between GPUs or gloo on the host).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import nis


def _pack(rgb: torch.Tensor, pix: torch.Tensor, rows: int) -> torch.Tensor:
    """rgb (k, 3) float32 and pix (k,) int32 -> one (rows, 4) int32 payload: the radiance's
    bits in columns 0-2, the pixel index in column 3, rows past k set to -1 (no pixel)."""
    k = int(pix.shape[0])
    out = torch.full((rows, 4), -1, dtype=torch.int32, device=pix.device)
    if k:
        out[:k, :3] = rgb[:k].contiguous().view(torch.int32)
        out[:k, 3] = pix[:k]
    return out


def _unpack(payload: torch.Tensor, k: int) -> tuple[torch.Tensor, torch.Tensor]:
    rgb = payload[:k, :3].contiguous().view(torch.float32)
    pix = payload[:k, 3].contiguous()
    return rgb, pix


def gather_parts(rgb: torch.Tensor, pix: torch.Tensor, rows: int, dst: int = 0, group=None):
    """Gathers every rank's part (rgb (k, 3) float32, pix (k,) int32, k <= rows) to rank
    `dst`.  Returns the list of (rgb, pix) in rank order on `dst`, None on the others.

    All ranks pass the same `rows`; the payload is rows x 16 bytes per rank whatever k is,
    and the counts travel in a separate gather of one int64 per rank."""
    if int(pix.shape[0]) > rows or int(rgb.shape[0]) < int(pix.shape[0]):
        raise ValueError("part larger than the agreed row count, or fewer rgb rows than pixels")
    if not (dist.is_available() and dist.is_initialized()):
        return [(rgb[:int(pix.shape[0])], pix)]        # one process: its part is the frame
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    dev = pix.device
    count = torch.tensor([int(pix.shape[0])], dtype=torch.int64, device=dev)
    payload = _pack(rgb, pix, rows)
    counts = [torch.empty_like(count) for _ in range(world)] if rank == dst else None
    bufs = [torch.empty_like(payload) for _ in range(world)] if rank == dst else None
    dist.gather(count, counts, dst=dst, group=group)
    dist.gather(payload, bufs, dst=dst, group=group)
    if rank != dst:
        return None
    return [_unpack(b, int(c.item())) for b, c in zip(bufs, counts)]


def render_frame_split(ctx: nis.Context, vol: int, light: int, weights: int, mat: dict,
                       cam: dict, dst: int = 0, group=None, stream=None, out=None,
                       part_bufs=None):
    """The frame of ``ctx.render_frame`` with its shading points split over the ranks of
    `group` (one process, no process group: the whole frame).  Returns (image, info) on `dst`
    (image (height, width, 3) float32 on ctx's device; `out` if given) and (None, info)
    elsewhere; info = dict(n_hits, first, count, rows).  part_bufs = (rgb, pix) device
    buffers of nis.part_capacity(width * height, world) rows, reused across frames."""
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    prgb, ppix = part_bufs if part_bufs is not None else (None, None)
    rgb, pix, n_hits, first = ctx.render_frame_part(vol, light, weights, mat, cam, rank, world,
                                                    rgb=prgb, pix=ppix, stream=stream)
    rows = nis.part_capacity(n_hits, world)     # the largest range of n_hits split world ways
    parts = gather_parts(rgb, pix, max(rows, 1), dst=dst, group=group)
    info = {"n_hits": n_hits, "first": first, "count": int(pix.shape[0]), "rows": rows}
    if parts is None:
        return None, info
    image = out if out is not None else torch.empty(
        (int(cam["height"]), int(cam["width"]), 3), dtype=torch.float32, device=pix.device)
    image.zero_()
    for r, p in parts:
        ctx.scatter_part(r, p, image, stream=stream)
    return image, info
