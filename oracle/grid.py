"""Cell masks of the block-structured grid with 2:1 time-nested refinement.

The domain is cut into blocks of 8^3 cells (the hybrid block structure of
Section 1 and Section 3.2).  Level l+1 covers the refined blocks of level l,
each split into 8 child blocks, with grid spacing and time step halved
(nested time stepping, Section 3.2).  The interface treatment follows
Yu et al. as cited in Sections 1 and 3.2; the paper does not write it out,
so this module fixes the following cell-centred reading:

* active_l   cells of level-l blocks that are not refined;
* hidden1_l  refined cells at Chebyshev distance 1 from an active cell,
  hidden2_l  at distance 2 (they hold the restriction of the finer level);
* ghost_l    (l >= 1) cells outside the level-l blocks at Chebyshev distance 1
  from them (they receive the coarse-to-fine interpolation);
* update_l = active_l | hidden1_l is what one stream-collide pass touches.

Masks are (NZ, NY, NXp) with NXp = NX + 2 when x is not periodic: padded
x index 0 is the inflow ghost column (x = -1) and NX + 1 the outflow column.
"""
import torch

BLOCK = 8


def _dilate(mask, periodic_x):
    """Chebyshev-1 dilation with wrap in y, z (and x when periodic).

    With padded x the wrap only moves data between the two ghost columns,
    which never hold region cells, so torch.roll is exact here.
    """
    out = mask.clone()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == dy == dx == 0:
                    continue
                out |= torch.roll(mask, shifts=(dz, dy, dx), dims=(0, 1, 2))
    return out


def _cells(block_mask, periodic_x):
    """Expand a (nbz, nby, nbx) block mask to cells, padding x if needed."""
    c = block_mask.repeat_interleave(BLOCK, 0).repeat_interleave(BLOCK, 1) \
        .repeat_interleave(BLOCK, 2)
    if not periodic_x:
        c = torch.nn.functional.pad(c, (1, 1))
    return c


class Level:
    """Masks and sizes of one refinement level."""

    def __init__(self, l, nb, periodic_x, region_blocks, refine_blocks):
        self.l = l
        self.nbx, self.nby, self.nbz = (n << l for n in nb)
        self.NX, self.NY, self.NZ = BLOCK * self.nbx, BLOCK * self.nby, BLOCK * self.nbz
        self.periodic_x = periodic_x
        self.xoff = 0 if periodic_x else 1
        self.region_blocks = region_blocks
        self.refine_blocks = refine_blocks
        self.region = _cells(region_blocks, periodic_x)
        self.refined = _cells(refine_blocks, periodic_x)
        self.active = self.region & ~self.refined
        d1 = _dilate(self.active, periodic_x)
        d2 = _dilate(d1, periodic_x)
        self.hidden1 = self.refined & d1
        self.hidden2 = self.refined & d2 & ~d1
        inside = torch.zeros_like(self.region)
        inside[:, :, self.xoff:self.xoff + self.NX] = True
        self.ghost = _dilate(self.region, periodic_x) & ~self.region & inside \
            if l > 0 else torch.zeros_like(self.region)
        self.update = self.active | self.hidden1
        self.valid = self.active | self.hidden1 | self.hidden2


def block_dilate(b, periodic_x):
    """Chebyshev-1 dilation of a block mask (same wrap rules as cells, but the
    block grid has no padding so non-periodic x must not wrap)."""
    out = b.clone()
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz == dy == dx == 0:
                    continue
                r = torch.roll(b, shifts=(dz, dy, dx), dims=(0, 1, 2))
                if not periodic_x and dx != 0:
                    if dx == 1:
                        r[:, :, 0] = False
                    else:
                        r[:, :, -1] = False
                out |= r
    return out


def build_levels(nb, periodic_x, refine):
    """Levels from coarse block counts nb = (nbx, nby, nbz) and refine flags.

    refine: list of bool tensors, refine[l] of shape (nbz*2^l, nby*2^l, nbx*2^l),
    one per level except the finest.  Checks the nesting rule that every
    block touching a refined block of level l >= 1 belongs to level l, so the
    interpolation stencils of the next level see only level-l cells.
    """
    nbx, nby, nbz = nb
    region = torch.ones(nbz, nby, nbx, dtype=torch.bool)
    levels = []
    for l in range(len(refine) + 1):
        ref = refine[l].bool() if l < len(refine) else torch.zeros_like(region)
        if ref.shape != region.shape:
            raise ValueError("refine[%d] has shape %s, expected %s"
                             % (l, tuple(ref.shape), tuple(region.shape)))
        if bool((ref & ~region).any()):
            raise ValueError("refine flag on a block outside level %d" % l)
        if l > 0 and bool((block_dilate(ref, periodic_x) & ~region).any()):
            raise ValueError("refined block of level %d touches the level boundary" % l)
        if l + 1 < len(refine) + 1 and not bool(ref.any()):
            raise ValueError("level %d has no refined block" % l)
        levels.append(Level(l, nb, periodic_x, region, ref))
        region = ref.repeat_interleave(2, 0).repeat_interleave(2, 1).repeat_interleave(2, 2)
    return levels
