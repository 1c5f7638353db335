"""Replica runs on several GPUs of one node.

The method's data path does not shard here: each rank runs its own Markov
chain (its own seeded inputs) on its own GPU, with no collective on the data
path.  Only the measurement crosses ranks: a barrier around the timed region,
the maximum of the step time over ranks, and the sum of the work done.  The
process group uses NCCL with CUDA tensors on GPU runs and gloo with CPU
tensors otherwise (the multi-process tests).  Rendezvous from the usual
torchrun environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR/PORT).
"""
import os


class Replicas:
    def __init__(self, backend=None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
            if backend == "nccl":
                torch.cuda.set_device(self.local)
                self.device = f"cuda:{self.local}"
                dist.init_process_group("nccl", device_id=torch.device(self.device))
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def seed(self, base):
        """Input seed of this replica (independent chains per rank)."""
        return base + 100 * self.rank

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def allmax(self, x):
        """Maximum over ranks (the step time of the slowest replica)."""
        return self._reduce(x, self.dist.ReduceOp.MAX if self.dist else None)

    def allsum(self, x):
        """Sum over ranks (the work all replicas did)."""
        return self._reduce(x, self.dist.ReduceOp.SUM if self.dist else None)

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None
