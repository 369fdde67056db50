"""Row-sharded pass over several ranks, one GPU each (Eq. 11: the sketch is a sum over rows).

Each rank runs one session over its own share of the rows. The one exchange step gathers
every rank's checkpoint (the bytes of ``spca_save_state``) on the root rank, in rank order,
and merges them into the root's session with ``spca_merge``, which rebases each share onto
the root's shift c. The root session then holds the sketch of all rows and is the only one
that finalizes. torch.distributed carries the bytes: gloo between host processes, NCCL
between GPUs. The checkpoints are of the order of n (l + 1) doubles per rank; nothing else
crosses ranks.
"""
import torch
import torch.distributed as dist


def row_shard(m, world, rank, block):
    """Rows [r0, r1) of rank `rank`: whole blocks of `block` rows dealt out contiguously,
    the first (nblocks % world) ranks taking one block more; every row belongs to one rank."""
    nblk = (m + block - 1) // block
    base, extra = divmod(nblk, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return min(m, b0 * block), min(m, b1 * block)


def _device_for(group):
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_bytes(data, group=None, root=0):
    """Every rank's `data` (bytes) on `root`, in rank order (None on the other ranks)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = _device_for(group)
    size = torch.tensor([len(data)], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(size) for _ in range(world)]
    dist.all_gather(sizes, size, group=group)
    sizes = [int(s.item()) for s in sizes]
    width = max(sizes)
    buf = torch.zeros(width, dtype=torch.uint8, device=dev)
    if len(data):
        buf[:len(data)] = torch.frombuffer(bytearray(data), dtype=torch.uint8).to(dev)
    parts = [torch.empty(width, dtype=torch.uint8, device=dev) for _ in range(world)] if rank == root else None
    dist.gather(buf, parts, dst=root, group=group)
    if rank != root:
        return None
    return [bytes(p[:s].cpu().numpy().tobytes()) for p, s in zip(parts, sizes)]


def merge_blobs(session, blobs, root=0, scratch=None, merge=None):
    """Add the checkpoints `blobs` (one per rank, in rank order; root's own is skipped) into
    `session` through `scratch`, a session of the same parameters (load_state, then
    `merge(session, scratch)`; default spca_merge)."""
    if merge is None:
        from . import spca_merge

        def merge(dst, src):
            spca_merge(dst.handle, src.handle)
    for r, blob in enumerate(blobs):
        if r == root:
            continue
        scratch.load_state(blob)
        merge(session, scratch)


def merge_across_ranks(session, group=None, root=0, scratch=None, merge=None):
    """Sum every rank's session into root's (the exchange step of the row-sharded pass).

    `session` has save_state(); on root, `scratch` is a session of the same parameters that
    takes each other rank's checkpoint in turn (merge_blobs). Returns True on root, False
    elsewhere. Ranks merge in rank order, so the result does not depend on arrival order.
    """
    blobs = gather_bytes(session.save_state(), group=group, root=root)
    if blobs is None:
        return False
    merge_blobs(session, blobs, root=root, scratch=scratch, merge=merge)
    return True


def scratch_like(session):
    """An empty session with `session`'s parameters (the root's merge scratch)."""
    from . import Session
    return Session(session.n, session.k, session.p, session.seed, math=session.math, center=session.center,
                   max_block_rows=session.max_block_rows)
