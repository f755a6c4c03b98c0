"""Split one integration over ranks (one process per GPU) by range gates.

Gates are independent (each gate's spectrum needs only its own echo window, Eqs. 7-8), so
a rank can integrate a contiguous block of gates from the echo samples those gates read,
with no exchange during the integration; the [R_g][nfft] blocks are gathered at the end.
Host-side bookkeeping only: the integration itself is the plan's (``isr.Plan``).
"""
from __future__ import annotations


def gate_blocks(n_ranges: int, world: int) -> list[tuple[int, int]]:
    """Contiguous (first_gate, count) per rank; counts differ by at most one, the first
    ``n_ranges % world`` ranks take one gate more.  A rank may get zero gates only when
    ``world > n_ranges``."""
    if n_ranges < 0 or world < 1:
        raise ValueError("n_ranges must be >= 0 and world >= 1")
    base, extra = divmod(n_ranges, world)
    out, first = [], 0
    for r in range(world):
        c = base + (1 if r < extra else 0)
        out.append((first, c))
        first += c
    return out


def echo_span(first: int, count: int, range_start: int, range_step: int, code_len: int) -> dict:
    """Echo samples a block of gates reads, as a plan geometry on the sub-rows.

    The block's windows cover [s_first, s_last + code_len) with s_g = range_start + g step.
    The sub-row starts at ``s0`` = s_first rounded down to a multiple of 4 samples (16 bytes:
    the row alignment the plan requires) and is ``echo_stride`` samples long (a multiple of 4);
    the block's first gate starts at ``range_start`` = s_first - s0 within it.  The span never
    reaches past the original row's rounded end, so slicing [s0, s0 + echo_stride) of a row
    whose stride is a multiple of 4 stays inside it."""
    if count < 1:
        raise ValueError("a block needs at least one gate")
    s_first = range_start + first * range_step
    s_last = s_first + (count - 1) * range_step
    s0 = s_first - (s_first % 4)
    s1 = s_last + code_len
    stride = (s1 - s0 + 3) // 4 * 4
    return {"s0": s0, "s1": s1, "echo_stride": stride, "range_start": s_first - s0}


def gather_gate_blocks(local, blocks: list[tuple[int, int]], rank: int, world: int, dst: int = 0):
    """Gather every rank's [count][nfft] block into one [n_ranges][nfft] tensor on rank ``dst``
    (None elsewhere).  ``local`` lives where the process group's backend expects it (CUDA for
    NCCL, CPU for gloo); blocks are padded to the largest count for the collective and the
    padding is dropped.  With world == 1 this returns ``local`` itself."""
    import torch
    import torch.distributed as dist

    if world == 1:
        return local
    counts = [c for _, c in blocks]
    cmax = max(counts)
    nfft = local.shape[1]
    pad = torch.zeros((cmax, nfft), dtype=local.dtype, device=local.device)
    pad[:counts[rank]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)] if rank == dst else None
    dist.gather(pad, gather_list=bufs, dst=dst)
    if rank != dst:
        return None
    return torch.cat([b[:c] for b, c in zip(bufs, counts)], dim=0)
