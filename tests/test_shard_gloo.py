"""The split of the top recursion level over ranks (paper_2309_00628_gb300/shard.py), on CPU ranks.

Each gloo rank computes its top-level products' contribution with the oracle (the GPU ranks call
sw_mm_products instead), the C quadrants are reduced onto their owners and broadcast back; the
result must equal the exact product on integer inputs, for 2, 3 and 8 ranks (8 > 7 products:
a rank with no product still takes part in the reduction), with and without the final gather,
and for rectangular odd shapes (zero padding, Sec. 3.1).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, cases, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2309_00628_gb300 import inputs, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for (m, n, k, cutoff, alg, gather) in cases:
            A, B = inputs.pair(m, n, k, "int", seed=21, dtype=np.float64, lim=4)
            L = oracle.depth(m, n, k, cutoff)
            s = 1 << L
            block = (-(-m // s) * (s // 2), -(-n // s) * (s // 2))  # the padded top-level quadrants

            def partial(a, b, c, v, mask):
                return torch.from_numpy(oracle.recursive_products(alg, a, b, c, mask))

            C = shard.sharded_mm(A, B, cutoff, 0, partial, gather=gather, block=block)
            res.append(C.numpy())
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def _run(world, cases):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3, 8])
def test_sharded_product_matches_the_exact_product(world):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2309_00628_gb300 import inputs, shard
    cases = [(32, 32, 32, 8, oracle.WINOGRAD, True), (37, 22, 45, 5, oracle.STRASSEN, True),
             (24, 40, 16, 4, oracle.KNUTH, True), (32, 32, 32, 8, oracle.WINOGRAD, False)]
    res = _run(world, cases)
    for i, (m, n, k, cutoff, alg, gather) in enumerate(cases):
        A, B = inputs.pair(m, n, k, "int", seed=21, dtype=np.float64, lim=4)
        ex = A.astype(np.int64) @ B.astype(np.int64)
        L = oracle.depth(m, n, k, cutoff)
        s = 1 << L
        bm, bn = -(-m // s) * (s // 2), -(-n // s) * (s // 2)
        for r in range(world):
            C = res[r][i]
            if gather:
                assert np.array_equal(C, ex), (world, r, i)
            else:  # each owner holds its own quadrants
                for q, ((r0, r1), (c0, c1)) in enumerate(shard.quadrant_slices(m, n, bm, bn)):
                    if shard.quadrant_owner(q, world) == r:
                        assert np.array_equal(C[r0:r1, c0:c1], ex[r0:r1, c0:c1]), (world, r, q)


def test_product_masks_cover_each_product_once():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2309_00628_gb300 import shard
    for world in range(1, 10):
        masks = shard.product_masks(world)
        assert len(masks) == world
        tot = 0
        for msk in masks:
            assert tot & msk == 0
            tot |= msk
        assert tot == 0x7F
        counts = [bin(msk).count("1") for msk in masks]
        assert max(counts) - min(counts) <= 1
