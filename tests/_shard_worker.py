"""One rank of the sharded-oracle check (run by tests/test_sharding.py, never collected).

Reads RANK, WORLD_SIZE, MASTER_ADDR, MASTER_PORT from the environment, joins a gloo
process group, takes its shard of subjects from libcopa's partitioner, runs the oracle's
sharded outer iteration (oracle/sharded.py) with torch.distributed.all_reduce as the sum
over shards, and saves its state and FIT history to the .npz path given as argv[1]."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import paper_1803_04572_gb300 as P  # noqa: E402
import synth  # noqa: E402
from oracle import copa_oracle as O  # noqa: E402
from oracle import sharded as OS  # noqa: E402

from test_sharding import CASE, N_OUTER, OPT  # noqa: E402


def main():
    rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X, init = CASE()
    bounds = P.partition(X.subj_ptr, X.row_ptr, world)
    k0, k1 = int(bounds[rank]), int(bounds[rank + 1])
    Xs = X.subset(np.arange(k0, k1))
    st = OS.shard_state(O.State.from_init(*init), k0, k1)

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        dist.all_reduce(t)
        return t.numpy()

    fits = []
    for _ in range(N_OUTER):
        st, f = OS.outer_iteration(Xs, st, OPT, allreduce)
        fits.append(f)
    np.savez(sys.argv[1], H=st.H, V=st.V, W=st.W, DW=st.DW, fits=np.array(fits), bounds=bounds)
    dist.barrier()
    dist.destroy_process_group()


if __name__ == "__main__":
    main()
