"""The exchange of one scene's HR set split across ranks.

HR particles never act on one another (Sec. 4: an HR particle's update reads
the LR state and its own position and velocity only), so every rank runs the
whole LR computation and updates one slab of the cell-ordered HR slots
(``Context.set_hr_slab``).  Before each HR reorder, and before the HR state is
read in original order, the ranks exchange their slabs: one all-gather of
(position, velocity) slabs, after which every rank writes the whole state
back (``Context.hr_slab_assemble``) and all ranks hold the same bits.
"""
from . import gs_hr_slab_range


def slab_ranges(n_slots, n_parts):
    """The [begin, end) slot range of every part, from the library."""
    out = []
    for part in range(n_parts):
        rc, b, e = gs_hr_slab_range(n_slots, part, n_parts)
        if rc != 0:
            raise ValueError(f"no slab partition of {n_slots} slots into {n_parts} parts")
        out.append((b, e))
    return out


def all_gather_slabs(pos, vel, rank, world, group=None):
    """Every rank passes its whole (slots, 4) position and velocity tensors,
    of which only its own slab is current; on return both hold every rank's
    slab.  One all_gather of equal-sized (pos | vel) blocks, padded to the
    largest slab."""
    import torch
    import torch.distributed as dist
    n = pos.shape[0]
    ranges = slab_ranges(n, world)
    width = max(e - b for b, e in ranges)
    b, e = ranges[rank]
    mine = torch.zeros((width, 8), dtype=pos.dtype, device=pos.device)
    mine[: e - b, :4] = pos[b:e]
    mine[: e - b, 4:] = vel[b:e]
    blocks = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(blocks, mine, group=group)
    for r, (rb, re) in enumerate(ranges):
        pos[rb:re] = blocks[r][: re - rb, :4]
        vel[rb:re] = blocks[r][: re - rb, 4:]
    return pos, vel


def assemble(ctx, rank, world, group=None):
    """Gather-back for a Context restricted to slab `rank` of `world`: read
    its internal HR state into device tensors, exchange the slabs, write the
    whole state back."""
    import torch

    from . import GS_FIELD_HR_POS_INTERNAL, GS_FIELD_HR_VEL_INTERNAL
    pos = torch.empty((ctx.hr_slots, 4), dtype=torch.float32, device="cuda")
    vel = torch.empty_like(pos)
    ctx.read(GS_FIELD_HR_POS_INTERNAL, pos)
    ctx.read(GS_FIELD_HR_VEL_INTERNAL, vel)
    ctx.sync()
    all_gather_slabs(pos, vel, rank, world, group)
    torch.cuda.synchronize()
    ctx.hr_slab_assemble(pos, vel)
