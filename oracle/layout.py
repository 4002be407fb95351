"""Brute-force sparse block tables (oracle).

Reading of the sparse layout (Sec. 4 and Sec. 6.2; the paper orders blocks
along a space-filling curve and splits boundary from non-boundary blocks,
but names no curve and no ordering):

* the virtual box is cut into cubic blocks of edge B (8 by default);
* a block is active iff it holds at least one updated voxel (type fluid,
  regularized velocity or regularized pressure);
* a block is a boundary block iff it holds at least one regularized voxel
  (Sec. 6.2: bounce-back voxels do not make a block "boundary");
* numbering (memory-based grouping, Sec. 4): boundary blocks first, then
  non-boundary blocks; inside each group ascending Morton code of the block
  coordinate with x in the lowest bit (bit 3k = x_k, 3k+1 = y_k, 3k+2 = z_k);
* numbering (bitmask-based grouping, Sec. 4): every block in ascending
  Morton code, whatever its group; a per-block bit marks the boundary blocks
  (bit b % 32 of 32-bit word b // 32), and the boundary values are reached
  through a per-slot index (-1 or the rank of the regularized voxel in
  flag-scan order, x fastest) into a compact buffer;
* nbr[b][k], k = (dx+1) + 3(dy+1) + 9(dz+1), is the id of the block at
  (bx+dx, by+dy, bz+dz) (wrapped on periodic axes) or -1.

Everything here is computed by the most direct loops over block
coordinates; it is compared byte for byte with the library's tables.
"""
import numpy as np

UPDATED_TYPES = (0, 2, 3)
REGULARIZED_TYPES = (2, 3)


def morton_code(bx, by, bz, bits=10):
    """Interleave the bits of (bx, by, bz), x in the lowest position."""
    code = 0
    for k in range(bits):
        code |= ((bx >> k) & 1) << (3 * k)
        code |= ((by >> k) & 1) << (3 * k + 1)
        code |= ((bz >> k) & 1) << (3 * k + 2)
    return code


def block_tables(flags, block_edge=8, periodic=(False, False, False), grouping="memory"):
    """Return dict(coords (n,3) int32, n_boundary, nbr (n,27) int32, ...).

    ``flags`` has shape (nz, ny, nx); the box is padded with type 7 (not in
    domain) up to a whole number of blocks.  grouping "memory" or "bitmask";
    the latter also returns boundary_bits (uint32 words) and bc_index (int32
    per slot, slot = b * B^3 + lx + B (ly + B lz)).
    """
    nz, ny, nx = flags.shape
    B = block_edge
    nbz, nby, nbx = -(-nz // B), -(-ny // B), -(-nx // B)
    types = flags & 7
    active, boundary = [], []
    for bz in range(nbz):
        for by in range(nby):
            for bx in range(nbx):
                t = types[bz * B:(bz + 1) * B, by * B:(by + 1) * B, bx * B:(bx + 1) * B]
                if np.isin(t, UPDATED_TYPES).any():
                    is_b = bool(np.isin(t, REGULARIZED_TYPES).any())
                    active.append((bx, by, bz))
                    boundary.append(is_b)
    if grouping == "memory":
        keys = [(0 if isb else 1, morton_code(*c)) for c, isb in zip(active, boundary)]
    elif grouping == "bitmask":
        keys = [morton_code(*c) for c in active]
    else:
        raise ValueError(grouping)
    order = sorted(range(len(active)), key=lambda i: keys[i])
    coords = np.array([active[i] for i in order], dtype=np.int32).reshape(-1, 3)
    n_boundary = int(sum(boundary))
    index = {tuple(int(v) for v in c): b for b, c in enumerate(coords)}
    nbr = np.full((len(coords), 27), -1, dtype=np.int32)
    dims_b = (nbx, nby, nbz)
    for b, c in enumerate(coords):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                    q = [int(c[0]) + dx, int(c[1]) + dy, int(c[2]) + dz]
                    ok = True
                    for a in range(3):
                        if q[a] < 0 or q[a] >= dims_b[a]:
                            if periodic[a]:
                                q[a] %= dims_b[a]
                            else:
                                ok = False
                    if ok:
                        nbr[b, k] = index.get(tuple(q), -1)
    out = {"coords": coords, "n_boundary": n_boundary, "nbr": nbr, "dims_blocks": dims_b}
    if grouping == "bitmask":
        is_b = [boundary[i] for i in order]
        words = np.zeros((len(coords) + 31) // 32, dtype=np.uint32)
        for b, v in enumerate(is_b):
            if v:
                words[b // 32] |= np.uint32(1 << (b % 32))
        bc_index = np.full(len(coords) * B ** 3, -1, dtype=np.int32)
        rank = 0
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if types[z, y, x] in REGULARIZED_TYPES:
                        b = index[(x // B, y // B, z // B)]
                        bc_index[b * B ** 3 + (x % B) + B * ((y % B) + B * (z % B))] = rank
                        rank += 1
        out["boundary_bits"] = words
        out["bc_index"] = bc_index
    return out


def multires_tables(level_map, n_levels, cell, block_edge=8, q=19):
    """Brute-force multi-resolution block tables (periodic box).

    Reading (Sec. 5; Sec. 6.3): level l owns the regions the level map gives
    it; each level is cut into blocks of block_edge voxels of that level.  A
    voxel has distance 0 (property P_d) iff one of its neighbours along the
    lattice's velocities (D3Q19, or D3Q27 with q = 27) is owned by another
    level; a block is G_c iff it holds such a voxel, else
    G_i.  Numbering per level: G_c blocks first, then G_i, each in Morton
    order.  Returns one dict per level with coords, n_c, nbr (27 same-level
    neighbours, -1 = none), xnbr_coarse (27: level-(l+1) block covering the
    neighbour region, else -1) and xnbr_fine (27 x 8: the level-(l-1) blocks
    covering the neighbour region, octant j = x + 2y + 4z, else -1).
    """
    from .lattice import lattice
    C = lattice(q).C
    level_map = np.asarray(level_map)
    B = block_edge
    own = []
    for lv in range(n_levels):
        r = cell // (2 ** lv)
        own.append(level_map.repeat(r, 0).repeat(r, 1).repeat(r, 2))
    out = []
    bmaps = []
    for lv in range(n_levels):
        o = own[lv]
        dist0 = np.zeros(o.shape, bool)
        for i in range(1, len(C)):
            cx, cy, cz = (int(v) for v in C[i])
            dist0 |= np.roll(o, shift=(cz, cy, cx), axis=(0, 1, 2)) != lv
        dist0 &= o == lv
        nz, ny, nx = o.shape
        nbz, nby, nbx = nz // B, ny // B, nx // B
        rows = []
        for bz in range(nbz):
            for by in range(nby):
                for bx in range(nbx):
                    sl = (slice(bz * B, (bz + 1) * B), slice(by * B, (by + 1) * B),
                          slice(bx * B, (bx + 1) * B))
                    if (o[sl] == lv).any():
                        gc = bool(dist0[sl].any())
                        rows.append(((0 if gc else 1, morton_code(bx, by, bz)), (bx, by, bz), gc))
        rows.sort(key=lambda r: r[0])
        coords = np.array([r[1] for r in rows], dtype=np.int32).reshape(-1, 3)
        bmap = {tuple(int(v) for v in c): b for b, c in enumerate(coords)}
        bmaps.append(bmap)
        out.append({"coords": coords, "n_c": sum(1 for r in rows if r[2]),
                    "dims_blocks": (nbx, nby, nbz)})
    for lv in range(n_levels):
        t = out[lv]
        nbx, nby, nbz = t["dims_blocks"]
        nb = len(t["coords"])
        nbr = np.full((nb, 27), -1, np.int32)
        xc = np.full((nb, 27), -1, np.int32)
        xf = np.full((nb, 27, 8), -1, np.int32)
        for b, c in enumerate(t["coords"]):
            for k in range(27):
                dx, dy, dz = k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1
                q = ((int(c[0]) + dx) % nbx, (int(c[1]) + dy) % nby, (int(c[2]) + dz) % nbz)
                nbr[b, k] = bmaps[lv].get(q, -1)
                owner = own[lv][q[2] * B, q[1] * B, q[0] * B]
                if owner == lv + 1:
                    xc[b, k] = bmaps[lv + 1][(q[0] // 2, q[1] // 2, q[2] // 2)]
                elif owner == lv - 1:
                    for j in range(8):
                        f = (2 * q[0] + (j & 1), 2 * q[1] + ((j >> 1) & 1), 2 * q[2] + (j >> 2))
                        xf[b, k, j] = bmaps[lv - 1][f]
        t.update(nbr=nbr, xnbr_coarse=xc, xnbr_fine=xf)
    return out


def multires_interface(level_map, n_levels, cell, q=19):
    """Interface voxels of every level and the populations they read from
    another level's buffers (Sec. 5: voxels with P_d = 0; exchange as in
    oracle.multires, whose reading of the two-substep exchange it follows).

    Population i of a voxel G owned by level l is read from another level iff
      explosion:   the voxel G - c_i belongs to level l+1, or
      coalescence: one of the 8 subcells p of G reads level-(l-1) data in the
                   two virtual substeps, i.e. the level-(l-1) voxel p - c_i or
                   p - 2 c_i belongs to level l-1 (otherwise all 8 subcells
                   read G - c_i of level l and their mean is the plain pull).
    Returns one (slots, cross) pair per level: slot = block * 512 + x + 8 y +
    64 z (block ids of multires_tables, voxel inside the 8^3 block) in
    ascending order, cross = uint32 bit set of those populations.
    """
    from .lattice import lattice
    C = lattice(q).C
    level_map = np.asarray(level_map)
    tabs = multires_tables(level_map, n_levels, cell, q=q)
    own = []
    for lv in range(n_levels):
        r = cell // (2 ** lv)
        own.append(level_map.repeat(r, 0).repeat(r, 1).repeat(r, 2))

    def at(a, c, k):  # value at x - k c, periodic (axes z, y, x)
        return np.roll(a, shift=(k * int(c[2]), k * int(c[1]), k * int(c[0])), axis=(0, 1, 2))

    out = []
    for lv in range(n_levels):
        o = own[lv]
        cross = np.zeros(o.shape, np.uint32)
        for i in range(1, len(C)):
            dep = np.zeros(o.shape, bool)
            if lv + 1 < n_levels:
                dep |= at(o, C[i], 1) == lv + 1
            if lv > 0:
                fine = own[lv - 1] == lv - 1
                reads = at(fine, C[i], 1) | at(fine, C[i], 2)
                for j in range(8):
                    dep |= reads[(j >> 2)::2, ((j >> 1) & 1)::2, (j & 1)::2]
            cross |= np.where(dep & (o == lv), np.uint32(1 << i), np.uint32(0))
        bmap = {tuple(int(v) for v in c): b for b, c in enumerate(tabs[lv]["coords"])}
        zz, yy, xx = np.nonzero(cross)
        slots = np.array([bmap[(x // 8, y // 8, z // 8)] * 512 + (x % 8) + 8 * (y % 8) + 64 * (z % 8)
                          for x, y, z in zip(xx, yy, zz)], dtype=np.int64)
        order = np.argsort(slots, kind="stable")
        out.append((slots[order].astype(np.int32), cross[zz, yy, xx][order]))
    return out
