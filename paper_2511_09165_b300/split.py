"""One frame beamformed across several GPUs by directions.

Every (direction, sample) of a frame is independent, so a frame whose image is
too large for one GPU's time budget (the passive 8192-direction grids: 1 GiB
per image) splits along the directions: each rank owns a contiguous slice of
the direction grid and a plan for that slice only (its own delay table and
scratch on its own GPU).  Per frame:

  1. the frame, [N][T], is broadcast from the source rank to every rank (the
     only input every rank needs: the microphone signals do not depend on the
     direction);
  2. each rank beamforms its slice, [M_r][T], with its plan;
  3. the slices are gathered to the destination rank, which assembles the
     image [M][T] in the direction order of the grid.

The exchange is a broadcast and a gather through torch.distributed (NCCL for
CUDA tensors, gloo for host tensors); the beamforming itself is the library's
kernels on each rank.  A slice's plan groups its own directions, but a pixel's
sums run over the microphones in the same order whatever the grouping, so the
assembled image is bitwise that of one plan over the whole grid.
"""
from __future__ import annotations

import numpy as np


def direction_slices(n_dirs: int, world: int, align: int = 8) -> list[tuple[int, int]]:
    """Contiguous [lo, hi) slices of n_dirs directions for `world` ranks, as
    equal as whole groups of `align` directions allow (a rank may get none
    when there are fewer groups than ranks)."""
    if n_dirs < 0 or world < 1 or align < 1:
        raise ValueError("n_dirs >= 0, world >= 1 and align >= 1 are required")
    groups = (n_dirs + align - 1) // align
    out, lo_g = [], 0
    for r in range(world):
        hi_g = (groups * (r + 1)) // world
        lo, hi = min(lo_g * align, n_dirs), min(hi_g * align, n_dirs)
        out.append((lo, hi))
        lo_g = hi_g
    return out


def slice_grid(dir_azel=None, dir_unit=None, delays_s=None, lo: int = 0, hi: int = 0):
    """The rows [lo, hi) of whichever direction description is given."""
    def cut(a):
        return None if a is None else np.ascontiguousarray(np.asarray(a)[lo:hi])
    return cut(dir_azel), cut(dir_unit), cut(delays_s)


class SplitBeamformer:
    """This rank's share of a frame split by directions.

    rank, world : this process's rank and the number of ranks
    n_dirs      : directions of the whole grid
    beamform    : callable(frame, lo, hi) -> rows [hi - lo][T] for this
                  rank's slice (build it from a Plan over the slice: see
                  `plan_rows`); the frame it receives is on `device`
    group       : the torch.distributed process group (None: the default)
    """

    def __init__(self, rank: int, world: int, n_dirs: int, beamform, device=None,
                 group=None, align: int = 8):
        import torch
        self.torch = torch
        self.rank, self.world = int(rank), int(world)
        self.slices = direction_slices(int(n_dirs), self.world, align)
        self.lo, self.hi = self.slices[self.rank]
        self.rows = max(hi - lo for lo, hi in self.slices)
        self.n_dirs = int(n_dirs)
        self.beamform = beamform
        self.device = torch.device("cpu") if device is None else torch.device(device)
        self.group = group

    def __call__(self, frame, src: int = 0, dst: int = 0):
        """frame: [N][T] float32 on this rank's device (its values matter on
        `src` only).  Returns the image [M][T] on `dst`, None elsewhere."""
        import torch.distributed as td
        torch = self.torch
        td.broadcast(frame, src=src, group=self.group)
        T = frame.shape[1]
        part = torch.zeros((self.rows, T), dtype=torch.float32, device=self.device)
        if self.hi > self.lo:
            part[: self.hi - self.lo] = self.beamform(frame, self.lo, self.hi)
        # every rank sends the same shape (slices padded to the largest)
        parts = ([torch.empty_like(part) for _ in range(self.world)]
                 if self.rank == dst else None)
        td.gather(part, gather_list=parts, dst=dst, group=self.group)
        if self.rank != dst:
            return None
        image = torch.empty((self.n_dirs, T), dtype=torch.float32, device=self.device)
        for (lo, hi), p in zip(self.slices, parts):
            if hi > lo:
                image[lo:hi] = p[: hi - lo]
        return image


def plan_rows(plan):
    """The beamform callable of a SplitBeamformer for a Plan built over the
    rank's slice of the direction grid."""
    def run(frame, lo, hi):
        return plan(frame)
    return run
