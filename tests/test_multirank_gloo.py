"""The N > 1 host logic of bench.py on two CPU processes over gloo (no GPU):
each rank renders its own block of views of the same room (the data-parallel
split over views, with no collective on the data path), the timing is the
maximum over ranks and the barrier joins both."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), HM_BENCH_BACKEND="gloo")
    import bench
    from paper_2506_06988_b300 import scenes
    r, ws, _, dist = bench._dist()
    assert (r, ws) == (rank, world)
    t_max = bench._max_over_ranks(1.5 * (rank + 1), dist)
    bench._barrier(dist)
    s = scenes.room_scene(1, n_tris=2000, n_gauss=500, resolutions=((64, 48),) * 3, view_block=rank)
    poses = np.stack([np.concatenate([np.ravel(c.R), c.t]) for c in s.cameras])
    gathered = [None] * world
    dist.all_gather_object(gathered, (float(np.asarray(s.gaussians.means).sum()), poses))
    out[rank] = (t_max, gathered)
    dist.destroy_process_group()


def test_two_ranks_view_blocks_and_max_timing():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    from paper_2506_06988_b300 import scenes
    whole = scenes.room_scene(1, n_tris=2000, n_gauss=500, resolutions=((64, 48),) * 6)
    want = np.stack([np.concatenate([np.ravel(c.R), c.t]) for c in whole.cameras])
    for rank in range(world):
        t_max, gathered = res[rank]
        assert t_max == 3.0                                   # the slowest rank's time
        assert gathered[0][0] == gathered[1][0]                 # one scene on every rank
        assert not np.allclose(gathered[0][1], gathered[1][1])  # distinct views per rank
        # rank k's views are poses 3k..3k+2 of the scene's seeded pose sequence
        assert np.array_equal(gathered[0][1], want[:3]) and np.array_equal(gathered[1][1], want[3:])
