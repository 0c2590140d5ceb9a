"""Host checks of two arithmetic rules of the extraction kernels, restated in
numpy float32 with the kernels' operation order (each add, multiply and
divide rounded once, as the build's --fmad=false gives; fused multiply-adds
emulated with one rounding):

* the FP32 16-gon test of k_filter decides only where its error bound makes
  the decision the exact integer one: min over the edges F > 1 means strictly
  inside every edge, F < -1 on an edge means outside it (the hull filter of the
  boundary polygon, Sec. III.C);
* the transposed warp butterfly of the per-chunk sums gives the plain
  butterfly's totals bit for bit.
"""
import numpy as np

F32 = np.float32


def f32_of_int(c):
    """Round an integer to the nearest float32 (ties to even), exactly."""
    if c == 0:
        return F32(0.0)
    s, a = (-1 if c < 0 else 1), abs(c)
    nb = a.bit_length()
    if nb <= 24:
        return F32(s * a)
    sh = nb - 24
    q, r = divmod(a, 1 << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return F32(s * float(q) * 2.0 ** sh)


def fma32(a, b, c):
    """fma.rn.f32 on float32 arrays: a * b + c rounded once.  The product is
    exact in float64; the sum's rounding error comes from TwoSum, and a float64
    sum that lands exactly on a float32 rounding midpoint is resolved by the
    error's sign."""
    a, b, c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    # a midpoint between two adjacent float32 values is representable in float64
    lo = np.nextafter(r, F32(-np.inf)).astype(np.float64)
    hi = np.nextafter(r, F32(np.inf)).astype(np.float64)
    r64 = r.astype(np.float64)
    mid_dn = (r64 + lo) / 2.0
    mid_up = (r64 + hi) / 2.0
    r = np.where((s == mid_dn) & (e < 0), np.nextafter(r, F32(-np.inf)), r)
    r = np.where((s == mid_up) & (e > 0), np.nextafter(r, F32(np.inf)), r)
    return r.astype(np.float32)


def test_fma32_rounds_once():
    # 1 + 2^-24 is a float32 midpoint: the exact 1 + 2^-24 + 2^-60 rounds up, 1 + 2^-24 - 2^-60 down
    one = F32(1.0)
    assert fma32(F32(2.0 ** -30), F32(2.0 ** -30), fma32(one, one, F32(2.0 ** -24))) == F32(1.0)
    assert fma32(F32(2.0 ** -24), one, one) == one  # tie to even
    assert fma32(F32(2.0 ** -24) + F32(2.0 ** -47), one, one) == np.nextafter(one, F32(2))
    assert fma32(F32(3.0), F32(5.0), F32(-15.0)) == 0.0


def edges_of(poly, M):
    """The kernel's per-edge scaled lines (ex / E, -ey / E, -c / E) for a
    counter-clockwise polygon of integer vertices, M bounding |X|, |Y| + 1."""
    m = len(poly)
    out = []
    sM = F32(M)
    for i in range(m):
        (ax, ay), (bx, by) = poly[i], poly[(i + 1) % m]
        ex, ey = bx - ax, by - ay
        cc = ex * ay - ey * ax
        exf, eyf, cf = f32_of_int(ex), f32_of_int(ey), f32_of_int(cc)
        s = F32(abs(exf)) + F32(abs(eyf))
        E = F32(2.0) * (F32(0.5) * s + F32(4.76837158203125e-7) * (s * sM + F32(abs(cf))) + F32(1.0))
        out.append((exf / E, -(eyf / E), -(cf / E)))
    return out


def exact_cross(poly, X, Y):
    m = len(poly)
    res = []
    for i in range(m):
        (ax, ay), (bx, by) = poly[i], poly[(i + 1) % m]
        res.append((bx - ax) * (Y - ay) - (by - ay) * (X - ax))
    return np.stack(res)  # [edges, points], int64 (object for huge values)


def convex_poly(rng, center, radius, n=16):
    """A convex counter-clockwise polygon of n integer vertices on a
    perturbed circle (duplicates and collinear runs allowed, as the kernel's
    polygon of extremes can have)."""
    ang = np.sort(rng.uniform(0, 2 * np.pi, n))
    rad = radius * rng.uniform(0.7, 1.0, n)
    pts = np.stack([center[0] + rad * np.cos(ang), center[1] + rad * np.sin(ang)], 1)
    pts = np.round(pts).astype(np.int64)
    # convex hull (monotone chain) keeps it convex and ccw
    P = sorted(set(map(tuple, pts.tolist())))

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])
    lo, up = [], []
    for p in P:
        while len(lo) >= 2 and cross(lo[-2], lo[-1], p) <= 0:
            lo.pop()
        lo.append(p)
    for p in reversed(P):
        while len(up) >= 2 and cross(up[-2], up[-1], p) <= 0:
            up.pop()
        up.append(p)
    return lo[:-1] + up[:-1]


def near_edge_points(rng, poly, n_per_edge, spread):
    """Float plane coordinates (af, bf) within `spread` units of each edge's
    line (both sides), along the edge and past its ends."""
    out = []
    m = len(poly)
    for i in range(m):
        a, b = np.array(poly[i], float), np.array(poly[(i + 1) % m], float)
        e = b - a
        L = np.hypot(*e)
        if L == 0:
            continue
        nrm = np.array([-e[1], e[0]]) / L
        t = rng.uniform(-0.2, 1.2, n_per_edge)
        d = rng.uniform(-spread, spread, n_per_edge)
        p = a[None] + t[:, None] * e[None] + d[:, None] * nrm[None]
        out.append(p)
    return np.concatenate(out).astype(np.float32)


def classify(poly, pts):
    """(the kernel's keep flags, the exact keep flags, fast decisions taken)"""
    af, bf = pts[:, 0].astype(np.float32), pts[:, 1].astype(np.float32)
    X, Y = np.rint(af).astype(np.int64), np.rint(bf).astype(np.int64)
    M = float(max(np.abs(X).max(), np.abs(Y).max())) + 1.0
    ed = edges_of(poly, M)
    fmin = np.full(len(af), F32(2.0), np.float32)
    for (ex, ey, ez) in ed:
        fmin = np.minimum(fmin, fma32(ex, bf, fma32(ey, af, ez)))
    cr = exact_cross(poly, X, Y)
    exact_keep = ~np.all(cr > 0, axis=0)
    sure_in = fmin > F32(1.0)
    sure_out = fmin < F32(-1.0)
    # soundness of each fast decision
    assert not np.any(sure_in & exact_keep), "F > 1 on every edge but not strictly inside"
    if np.any(sure_out):
        # the edge where F < -1 has an exact cross product < 0
        for (ex, ey, ez), c in zip(ed, cr):
            f = fma32(ex, bf, fma32(ey, af, ez))
            assert np.all(c[f < F32(-1.0)] < 0), "F < -1 on an edge the point is not outside"
    keep = ~sure_in  # survivors and the band: the band takes the exact test
    band = keep & ~sure_out
    keep = np.where(band, exact_keep, keep)
    return keep, exact_keep, band


def test_polygon_filter_decisions_are_exact_near_edges():
    rng = np.random.default_rng(3)
    band_uniform = n_uniform = 0
    for trial in range(24):
        radius = [2.0e3, 6.0e4, 3.0e5, 2.0e6][trial % 4]
        center = rng.uniform(-radius, radius, 2)
        poly = convex_poly(rng, center, radius)
        if len(poly) < 3:
            continue
        pts = np.concatenate([near_edge_points(rng, poly, 200, 3.0),
                              near_edge_points(rng, poly, 50, 0.6),
                              (center + rng.uniform(-1.3 * radius, 1.3 * radius, (1500, 2))).astype(np.float32)])
        keep, exact, band = classify(poly, pts)
        assert np.array_equal(keep, exact)
        band_uniform += int(band[-1500:].sum())
        n_uniform += 1500
    # points spread over the cluster: the band around the edges holds a sliver of them
    assert band_uniform < 0.01 * n_uniform


def test_polygon_filter_at_the_largest_coordinates():
    # |X|, |Y| just under the 2^28 overflow guard: the bound grows with M and stays sound
    rng = np.random.default_rng(11)
    for trial in range(6):
        radius = 1.2e8
        center = rng.uniform(-1.0e8, 1.0e8, 2) * np.array([1, -1])[trial % 2]
        poly = convex_poly(rng, center, radius)
        pts = np.concatenate([near_edge_points(rng, poly, 150, 300.0),
                              (center + rng.uniform(-radius, radius, (600, 2))).astype(np.float32)])
        pts = np.clip(pts, -(2 ** 28) + 64, 2 ** 28 - 64).astype(np.float32)
        keep, exact, _ = classify(poly, pts)
        assert np.array_equal(keep, exact)


def butterfly(x):
    """Plain butterfly over 32 lanes: v += shfl_xor(v, s), s = 16 .. 1 (per value)."""
    v = x.copy()
    lanes = np.arange(32)
    s = 16
    while s:
        v = (v + v[lanes ^ s]).astype(np.float32)
        s >>= 1
    return v[0]  # every lane holds the same total


def transposed(x, P, L):
    """The kernel's transposed butterfly for values x[lane, e] (e < P): at level
    lv (offset 16 >> lv) a lane keeps half of its h * 2 values by its lane bit
    and adds its partner's copy of that half; then plain levels.  Returns the
    total of each value e, read from a lane whose top L bits equal e."""
    lanes = np.arange(32)
    cur = x.copy()  # [32, P]
    n = P
    for lv in range(L):
        s, h = 16 >> lv, n // 2
        up = (lanes & s) != 0
        keep = np.where(up[:, None], cur[:, h:n], cur[:, :h])
        send = np.where(up[:, None], cur[:, :h], cur[:, h:n])
        cur = (keep + send[lanes ^ s]).astype(np.float32)
        n = h
    v = cur[:, 0]
    s = 16 >> L
    while s:
        v = (v + v[lanes ^ s]).astype(np.float32)
        s >>= 1
    out = np.empty(P, np.float32)
    for e in range(P):
        lane = e << (5 - L)
        assert ((lane >> (5 - L)) & (P - 1)) == e
        out[e] = v[lane]
    return out


def test_transposed_warp_sums_equal_the_plain_butterfly():
    rng = np.random.default_rng(5)
    for P, L in ((4, 2), (8, 3)):
        for _ in range(200):
            # values of mixed magnitudes, so the association order matters
            x = (rng.standard_normal((32, P)) * 10.0 ** rng.integers(-3, 4, (32, P))).astype(np.float32)
            t = transposed(x, P, L)
            for e in range(P):
                assert t[e].tobytes() == butterfly(x[:, e]).tobytes()
