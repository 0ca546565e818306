"""Sample-sharded passes over several GPUs (one process per GPU).

The samples of a scan are independent (the paper spreads pointings over GPUs
x blocks x threads, Sec. 5.2), so a rank convolves a contiguous slice of the
pointing stream (contiguity keeps the disc reuse of consecutive samples) and
writes its own TOD slice: the forward pass needs no collective.  The
transposes do: the sky maps and the beam-grid gradient are sums over all
samples, so each rank's partial result is summed over the ranks with one
all-reduce (NCCL between GPUs; any torch.distributed backend works).
"""

import torch
import torch.distributed as dist


def shard_range(n, rank, world):
    """Contiguous slice [a, b) of n samples owned by ``rank`` of ``world``."""
    return n * rank // world, n * (rank + 1) // world


def _world(group):
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def allreduce_sum(*tensors, group=None):
    """Sum each tensor over the ranks of ``group`` in place (no-op on one rank)."""
    if _world(group) > 1:
        for t in tensors:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors if len(tensors) > 1 else tensors[0]


def sharded_adjoint(plan, theta, phi, psi, tod, det=0, group=None):
    """Sky maps (3, Npix) = A_S^T tod over all ranks' samples: each rank passes its own
    shard of the pointing and TOD, gets the transpose of the whole stream."""
    return allreduce_sum(plan.adjoint(theta, phi, psi, tod, det=det), group=group)


def sharded_adjoint_sky_beam(plan, theta, phi, psi, tod, det=0, group=None):
    """(maps, beam-grid gradient) over all ranks' samples (FP32 plans: one traversal each)."""
    maps, grad = plan.adjoint_sky_beam(theta, phi, psi, tod, det=det)
    return allreduce_sum(maps, grad, group=group)


def sharded_beam_grid_adjoint(plan, theta, phi, psi, y, det=0, tod=None, group=None):
    """Beam-grid gradient (6, N, N) over all ranks' samples.  With ``tod`` (this rank's
    forward TOD for the same samples) the Omega~(B_TT) term is added too: it is linear in
    sum_t y_t d_t, so each rank adds its own samples' share before the sum over ranks."""
    grad = plan.beam_grid_adjoint(theta, phi, psi, y, det=det)
    if tod is not None:
        plan.omega_adjoint(tod, y, grad, det=det)
    return allreduce_sum(grad, group=group)
