"""Split of the top recursion level over several GPUs (one process per GPU).

The seven products of one Strassen or Strassen-Winograd level (Sec. 2.2 P1..P7, Sec. 2.3 P1..P7)
are independent; only the post-additions combine them.  Rank r computes the products assigned to
it -- their contributions to C, through sw_mm_products on its own GPU, every level below the top
one as the one-GPU product -- and the ranks' contributions are then summed: each C quadrant is
reduced onto the rank that owns it and, if asked, the owners broadcast their quadrants so that
every rank holds C.  The exchange is the only collective of the path; the operands A and B are
replicated on every rank.

The reduction uses whatever torch.distributed backend the group was created with (NCCL on GPUs,
gloo on CPU tensors).  The per-rank computation is a parameter so that the exchange logic can be
exercised with CPU ranks; on GPUs it is `gpu_partial`, which runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
from typing import Callable, List, Optional

from . import swmm

NPRODUCTS = 7


def product_masks(world: int) -> List[int]:
    """Product p of the top level goes to rank p % world: masks (bit p) per rank.  With more ranks
    than products the extra ranks get the empty mask and only take part in the reduction."""
    if world < 1:
        raise ValueError("world must be >= 1")
    masks = [0] * world
    for p in range(NPRODUCTS):
        masks[p % world] |= 1 << p
    return masks


def quadrant_owner(q: int, world: int) -> int:
    """The rank a C quadrant (0: C11, 1: C12, 2: C21, 3: C22) is reduced onto."""
    return q % world


def quadrant_slices(m: int, n: int, block_m: int, block_n: int):
    """Row and column ranges of the four C quadrants of a top level with block sizes block_m x
    block_n (the last quadrant row / column takes what is left of m / n)."""
    rows = [(0, min(block_m, m)), (min(block_m, m), m)]
    cols = [(0, min(block_n, n)), (min(block_n, n), n)]
    return [(rows[q >> 1], cols[q & 1]) for q in range(4)]


def gpu_partial(h, A, B, cutoff: int, variant: int, mask: int, stream=None):
    """C_partial on this rank's GPU: the contributions of the top-level products in `mask`."""
    import torch
    assert A.is_cuda and B.is_cuda and A.dtype == B.dtype and A.dim() == 2 and B.dim() == 2
    m, k = A.shape
    n = B.shape[1]
    eb = 4 if A.dtype == torch.float32 else 8
    C = torch.empty((m, n), dtype=A.dtype, device=A.device)
    st = swmm.sw_mm_products(h, eb, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                             B.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(0), m, n, k, cutoff, variant,
                             mask, swmm._stream_ptr(stream))
    swmm.check(h, st)
    return C


def sharded_mm(A, B, cutoff: int, variant: int, partial: Callable, group=None, gather: bool = True,
               block=None):
    """C = A B with the top-level products split over the ranks of `group`.

    partial(A, B, cutoff, variant, mask) -> the rank's contribution (a tensor on the group's
    device type).  block = (block_m, block_n): the top level's quadrant sizes (default: halves,
    rounded up).  Returns C on every rank when gather is set, else each owner holds its quadrants
    (the rest of its tensor is its own partial)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mask = product_masks(world)[rank]
    C = partial(A, B, cutoff, variant, mask)
    m, n = C.shape
    bm, bn = block if block else ((m + 1) // 2, (n + 1) // 2)
    for q, ((r0, r1), (c0, c1)) in enumerate(quadrant_slices(m, n, bm, bn)):
        if r1 <= r0 or c1 <= c0:
            continue
        blk = C[r0:r1, c0:c1].contiguous()
        owner = quadrant_owner(q, world)
        dst = dist.get_global_rank(group, owner) if group is not None else owner
        dist.reduce(blk, dst=dst, op=dist.ReduceOp.SUM, group=group)
        if gather:
            dist.broadcast(blk, src=dst, group=group)
        if gather or rank == owner:
            C[r0:r1, c0:c1] = blk
    return C
