"""Host check of the one-pass CCL scheme the GPU runs (Algorithm 1 over
8^3 bricks, one pass per brick), on random vertex sets and random symmetric
edge predicates over the 26-neighbourhood: per brick, a union-find over the
brick and the cells its forward edges reach (x, y in -1..8, z in 0..8),
rooted at the smallest in-brick index; each brick vertex linked to its
component's root; each halo component, joined over the edges inside one
neighbour brick, joined to the root once.  Bricks are taken in random order.
The resulting partition must equal the one plain union over every edge
gives.  A variant that also joins halo cells over edges between two
different neighbour bricks is shown to lose edges, which is why the scheme
does not.  No GPU: the scheme is restated here in Python."""
import itertools

import numpy as np

FWD = [(1, dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)] + [(0, 1, dx) for dx in (-1, 0, 1)] + [(0, 0, 1)]


def _run(seed, same_brick, nb=(3, 3, 3), density=0.5, p_edge=0.7):
    rng = np.random.default_rng(seed)
    X, Y, Z = nb[0] * 8, nb[1] * 8, nb[2] * 8
    vert = rng.random((Z, Y, X)) < density
    salt = int(rng.integers(1 << 30))

    def gid(x, y, z):
        r = ((z // 8) * nb[1] + y // 8) * nb[0] + x // 8
        return r * 512 + ((z % 8) * 8 + y % 8) * 8 + x % 8

    def edge(a, b):  # a fixed pseudo-random draw per unordered pair
        a, b = min(a, b), max(a, b)
        return (hash((a, b, salt)) & 0xFFFF) < p_edge * 65536

    vs = [(x, y, z) for z in range(Z) for y in range(Y) for x in range(X) if vert[z, y, x]]
    # reference: plain union over every edge, smaller id as root
    ref = {gid(*v): gid(*v) for v in vs}

    def rfind(a):
        while ref[a] != a:
            a = ref[a]
        return a

    edges = {}
    for (x, y, z) in vs:
        for dz, dy, dx in FWD:
            x2, y2, z2 = x + dx, y + dy, z + dz
            if 0 <= x2 < X and 0 <= y2 < Y and z2 < Z and vert[z2, y2, x2]:
                e = edge(gid(x, y, z), gid(x2, y2, z2))
                edges[(gid(x, y, z), gid(x2, y2, z2))] = edges[(gid(x2, y2, z2), gid(x, y, z))] = e
                if e:
                    a, b = rfind(gid(x, y, z)), rfind(gid(x2, y2, z2))
                    if a != b:
                        ref[max(a, b)] = min(a, b)
    # the scheme, with a global forest that hooks the larger root under the smaller
    P = {gid(*v): gid(*v) for v in vs}

    def find(a):
        while P[a] != a:
            P[a] = P[P[a]]
            a = P[a]
        return a

    def union(a, b):
        a, b = find(a), find(b)
        if a != b:
            P[max(a, b)] = min(a, b)

    order = list(itertools.product(range(nb[0]), range(nb[1]), range(nb[2])))
    rng.shuffle(order)
    for bx, by, bz in order:
        cells = {}
        for hz in range(9):
            for hy in range(-1, 9):
                for hx in range(-1, 9):
                    x, y, z = bx * 8 + hx, by * 8 + hy, bz * 8 + hz
                    if 0 <= x < X and 0 <= y < Y and z < Z and vert[z, y, x]:
                        cells[(hx, hy, hz)] = gid(x, y, z)

        def inb(c):
            return 0 <= c[0] <= 7 and 0 <= c[1] <= 7 and c[2] <= 7

        def nbrick(c):
            return (c[0] // 8, c[1] // 8, c[2] // 8)

        def key(c):
            return ((c[2] * 8 + c[1]) * 8 + c[0]) if inb(c) else 512 + ((c[2] * 10 + c[1] + 1) * 10 + c[0] + 1)

        rp = {c: c for c in cells}
        hp = {c: c for c in cells}

        def f(F, a):
            while F[a] != a:
                a = F[a]
            return a

        def u(F, a, b):
            a, b = f(F, a), f(F, b)
            if a != b:
                if key(a) < key(b):
                    F[b] = a
                else:
                    F[a] = b

        for c in cells:
            for dz, dy, dx in FWD:
                c2 = (c[0] + dx, c[1] + dy, c[2] + dz)
                if c2 in cells and edges[(cells[c], cells[c2])]:
                    u(rp, c, c2)
                    if not inb(c) and not inb(c2) and (not same_brick or nbrick(c) == nbrick(c2)):
                        u(hp, c, c2)
        for c in cells:
            root = f(rp, c)
            if not inb(root):
                continue
            if inb(c):
                if root != c:
                    union(cells[c], cells[root])
            elif f(hp, c) == c:
                union(cells[c], cells[root])
    return sum(1 for v in P if find(v) != rfind(v))


def test_one_pass_scheme_reaches_the_plain_partition():
    for seed in range(9):
        assert _run(seed, True, density=[0.3, 0.5, 0.8][seed % 3], p_edge=[0.4, 0.7, 0.95][seed // 3]) == 0


def test_joining_halo_cells_across_two_neighbour_bricks_loses_edges():
    bad = [_run(seed, False, density=[0.3, 0.5, 0.8][seed % 3], p_edge=[0.4, 0.7, 0.95][seed // 3])
           for seed in range(9)]
    assert any(b > 0 for b in bad)
