"""Worker of the replica test: one rank of bench.py's host logic over gloo."""

import json
import os


def run(rank, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    import bench
    from workloads import make_batch

    dist.init_process_group("gloo", rank=rank, world_size=2)
    ws, r, _ = bench.dist_env()
    B, K, W = 8, 3, 2
    first = bench.rank_first_id(r, B, K, W)
    _, theta = make_batch(bench.WORKLOAD, B * K, first_id=first)
    t = bench.reduce_scalar(1.5 + r, "max", ws, torch.device("cpu"))
    conv = bench.reduce_scalar(100 + r, "sum", ws, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump({"ws": ws, "first": first, "theta0": theta[0].tolist(), "t": t, "conv": conv}, fh)
