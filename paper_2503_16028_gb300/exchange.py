"""Exchange step of a tempering layer with the particles sharded over ranks.

Rank r of R owns the contiguous block [lo_r, hi_r) of the N particles (block
sizes differ by at most one).  The particle move needs no exchange: every
particle's proposal, solve and accept test use only its own state (Alg. 2).
Once per tempering layer (Alg. 1) the ranks exchange:

1. the potentials: an all-gather of Phi, so that every rank finds the same
   next temperature by the ESS bisection and the same normalised weights;
2. nothing for the resampling indices: they depend on the global weights only,
   and the fixed-point CDF makes them independent of summation order, so every
   rank computes the same N indices from the gathered Phi;
3. the resampled particles: rank r needs the rows indices[lo_r:hi_r], wherever
   they live; `routing_plan` lists, for each (source, destination) pair, which
   local rows go where, and `exchange_rows` moves them point to point;
4. the mixture fit's sufficient statistics, summed over all particles: an
   all-reduce per EM iteration (`allreduce_sum`).

The functions take torch tensors and a torch.distributed process group: CPU
tensors over gloo or CUDA tensors over NCCL.  The arithmetic of each step runs
in the library on every rank; this module only moves data.
"""
import torch
import torch.distributed as dist


def block_bounds(n_total, world, rank):
    """[lo, hi) of rank's particles: blocks of n_total // world, the first n_total % world one larger."""
    q, rem = divmod(n_total, world)
    lo = rank * q + min(rank, rem)
    return lo, lo + q + (1 if rank < rem else 0)


def owner(i, n_total, world):
    """Rank that owns global particle i."""
    q, rem = divmod(n_total, world)
    big = rem * (q + 1)
    return i // (q + 1) if i < big else rem + (i - big) // q


def routing_plan(indices, n_total, world):
    """plan[src][dst] = (src_rows, dst_rows): global particle indices[j] for j in dst's block
    lives at local row src_rows[k] of src and goes to local row dst_rows[k] of dst (in the
    order of j, so the plan is the same on every rank)."""
    plan = [[([], []) for _ in range(world)] for _ in range(world)]
    for dst in range(world):
        lo, hi = block_bounds(n_total, world, dst)
        for j in range(lo, hi):
            i = int(indices[j])
            src = owner(i, n_total, world)
            slo, _ = block_bounds(n_total, world, src)
            plan[src][dst][0].append(i - slo)
            plan[src][dst][1].append(j - lo)
    return plan


def allgather_rows(local, n_total, group=None):
    """All ranks' blocks of rows concatenated in rank order (an all-gather of uneven blocks,
    padded to the largest block)."""
    world = dist.get_world_size(group)
    width = max(block_bounds(n_total, world, r)[1] - block_bounds(n_total, world, r)[0] for r in range(world))
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = []
    for r in range(world):
        lo, hi = block_bounds(n_total, world, r)
        out.append(parts[r][: hi - lo])
    return torch.cat(out, dim=0)


def exchange_rows(local, indices, n_total, group=None):
    """The rows indices[lo:hi] of the global particle array, for this rank's block [lo, hi),
    gathered from their owners by point-to-point messages (one per nonempty (src, dst))."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    plan = routing_plan(indices, n_total, world)
    lo, hi = block_bounds(n_total, world, rank)
    out = torch.empty((hi - lo,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    reqs, bufs = [], []
    for dst in range(world):                       # sends of my rows
        src_rows, _ = plan[rank][dst]
        if dst == rank or not src_rows:
            continue
        buf = local[torch.tensor(src_rows, device=local.device)].contiguous()
        bufs.append(buf)
        reqs.append(dist.isend(buf, dst, group=group, tag=rank))
    recvs = []
    for src in range(world):                       # receives of rows I need
        _, dst_rows = plan[src][rank]
        if src == rank or not dst_rows:
            continue
        buf = torch.empty((len(dst_rows),) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
        reqs.append(dist.irecv(buf, src, group=group, tag=src))
        recvs.append((buf, dst_rows))
    src_rows, dst_rows = plan[rank][rank]          # rows that stay
    if src_rows:
        out[torch.tensor(dst_rows, device=local.device)] = local[torch.tensor(src_rows, device=local.device)]
    for r in reqs:
        r.wait()
    for buf, rows in recvs:
        out[torch.tensor(rows, device=local.device)] = buf
    return out


def allreduce_sum(t, group=None):
    """In-place sum over ranks (the EM sufficient statistics of each rank's particles)."""
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
