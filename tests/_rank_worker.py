"""Worker of the multi-process bench test (spawned; one per rank)."""
import os


def job_rate_worker(rank, world, port, queue):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 100.0 + 50.0 * rank          # the highest rank is the slowest
        queue.put((rank, bench.max_over_ranks(ms), bench.job_rate(8, ms), bench.dist_env()))
    finally:
        dist.destroy_process_group()
