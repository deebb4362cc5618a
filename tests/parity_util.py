"""Helpers of the GPU-vs-oracle parity tests (host side only)."""
from __future__ import annotations

import numpy as np

import oracle

TOL_MAX_ABS = 2e-3   # per-pixel RGB(A) bound on non-boundary pixels (FP32 path)
TOL_PSNR_DB = 60.0   # over all pixels


def rect_fmin(u, v, A, B, C, x0, x1, y0, y1):
    """FP64 minimum of A dx^2 + 2 B dx dy + C dy^2 over the rectangle spanned
    by the pixel centres [x0, x1] x [y0, y1] (inclusive pixel indices),
    d = point - (u, v).  Vectorised over splats."""
    u, v, A, B, C = (np.asarray(t, np.float64) for t in (u, v, A, B, C))
    a1, a2 = np.asarray(x0) + 0.5 - u, np.asarray(x1) + 0.5 - u
    b1, b2 = np.asarray(y0) + 0.5 - v, np.asarray(y1) + 0.5 - v

    def edge(P, Q, R, a, lo, hi):
        t = np.clip(-Q * a / R, lo, hi)
        return P * a * a + 2 * Q * a * t + R * t * t

    f = np.minimum.reduce([edge(A, B, C, a1, b1, b2), edge(A, B, C, a2, b1, b2),
                           edge(C, B, A, b1, a1, a2), edge(C, B, A, b2, a1, a2)])
    inside = (a1 <= 0) & (a2 >= 0) & (b1 <= 0) & (b2 >= 0)
    return np.where(inside, 0.0, f)


def unreachable(p, g, W, H, slack):
    """True where splat g (oracle projection p) has no pixel centre of its
    box with alpha >= 1/255 (up to `slack` in the exponent)."""
    u, v = p["uv"][g, 0], p["uv"][g, 1]
    r = p["radius"][g]
    x0 = np.maximum(0, np.ceil(u - r - 0.5)); x1 = np.minimum(W - 1, np.floor(u + r - 0.5))
    y0 = np.maximum(0, np.ceil(v - r - 0.5)); y1 = np.minimum(H - 1, np.floor(v + r - 0.5))
    con = p["conic"][g]
    f = rect_fmin(u, v, con[:, 0], con[:, 1], con[:, 2], x0, x1, y0, y1)
    o = p["opacity"][g]
    with np.errstate(divide="ignore"):
        cut = 2 * np.log(255.0 * o)
    return (f > cut - 2 * slack) | (o * 255.0 < 1.0)


def splat_ids(r):
    """(instance, gaussian, template, level) of every GPU splat id."""
    groups = r.debug("groups")
    vis = r.debug("visible")
    S = int(sum(int(g[3]) * int(g[4]) for g in groups))
    inst = np.full(S, -1, np.int64)
    gau = np.full(S, -1, np.int64)
    lvl = np.full(S, -1, np.int64)
    for tpl, lv, slot0, nslots, ng, splat0, _block0 in groups:
        s = np.arange(int(nslots) * int(ng))
        inst[splat0 + s] = vis[slot0 + s // ng]
        gau[splat0 + s] = s % ng
        lvl[splat0 + s] = lv
    return inst, gau, lvl


def gpu_live(r, S):
    order = r.debug("depth_order").astype(np.int64)
    keys = r.debug("depth_keys")
    live = np.zeros(S, bool)
    live[order] = keys != 0xFFFFFFFF
    return live


def compare_splats(r, sc, os_=None, max_instances=None, instances=None):
    """Per-splat errors of the GPU records against the oracle, over GPU
    splats whose instance the oracle also projects.  Returns a dict of
    maxima and the per-splat arrays used for the tile-list checks."""
    os_ = os_ or oracle.OracleScene(sc)
    rec = r.debug("records").astype(np.float64)
    S = rec.shape[0]
    inst, gau, lvl = splat_ids(r)
    live = gpu_live(r, S)
    out = dict(duv=0.0, conic_rel=0.0, depth_rel=0.0, drgb=0.0, radius_mismatch=0, radius_boundary=0,
               live_mismatch=0, n=0, culled_unreachable=0)
    W, H = sc.camera.width, sc.camera.height
    insts = np.unique(inst)
    if instances is not None:
        insts = np.intersect1d(insts, np.asarray(list(instances), np.int64))
    if max_instances is not None:
        insts = insts[:max_instances]
    ref = {}
    for i in insts:
        p = oracle.project_instance(os_, int(i))
        ref[int(i)] = p
        m = np.nonzero(inst == i)[0]
        g = gau[m]
        ok_o = p["valid"][g] == 1
        ok_g = live[m]
        both = ok_o & ok_g
        # the GPU also drops splats no pixel of which reaches alpha 1/255;
        # anything else live on one side only is a boundary case (counted)
        dropped = ok_o & ~ok_g
        if dropped.any():
            un = unreachable(p, g[dropped], W, H, slack=1e-3)
            out["culled_unreachable"] += int(un.sum())
            out["live_mismatch"] += int((~un).sum())
        out["live_mismatch"] += int((~ok_o & ok_g).sum())
        if not both.any():
            continue
        mm, gg = m[both], g[both]
        R = rec[mm]
        duv = np.abs(R[:, 0:2] - p["uv"][gg]).max()
        con = np.stack([R[:, 2], R[:, 3], R[:, 4]], 1)
        cr = (np.abs(con - p["conic"][gg]) / np.maximum(np.abs(p["conic"][gg]).max(1, keepdims=True), 1e-30)).max()
        dr = (np.abs(R[:, 7] - p["depth"][gg]) / np.abs(p["depth"][gg])).max()
        drgb = np.abs(R[:, 8:11] - p["rgb"][gg]).max()
        rad_g = R[:, 6].astype(np.int64)
        rad_o = p["radius"][gg]
        mis = rad_g != rad_o
        near_int = np.abs(p["r_exact"][gg] - np.round(p["r_exact"][gg])) < 1e-3
        out["radius_mismatch"] += int(mis.sum())
        out["radius_boundary"] += int((mis & ~near_int).sum())
        out["duv"] = max(out["duv"], float(duv))
        out["conic_rel"] = max(out["conic_rel"], float(cr))
        out["depth_rel"] = max(out["depth_rel"], float(dr))
        out["drgb"] = max(out["drgb"], float(drgb))
        out["n"] += int(both.sum())
    out["ref"] = ref
    out["inst"], out["gau"], out["live"], out["rec"] = inst, gau, live, rec
    return out


def eps_from(errs) -> "oracle._Eps":
    """Boundary windows from measured per-splat errors: 4x each error (floors
    keep them positive).  The exponent window bounds |dq| <= 6.1 |duv| +
    5.6 |dQ|/|Q| for the exponents that matter (|q| <= ln 255 + 0.1, conic
    eigenvalues <= 1/0.3)."""
    duv = max(errs["duv"], 1e-6)
    cr = max(errs["conic_rel"], 1e-8)
    return oracle.default_eps(px=4 * duv + 1e-6, q=4 * (6.1 * duv + 5.6 * cr) + 1e-6,
                              radius=max(4 * 0.5 * cr * 100.0, 1e-5),
                              depth_rel=max(4 * errs["depth_rel"], 1e-7), near_z=1e-5)


def compare_images(got, ref):
    """got [H,W,4] float32 (GPU), ref: oracle.render output.  Returns a
    report dict."""
    g = np.asarray(got, np.float64)
    d = np.abs(g - ref["rgba"])
    boundary = ref["flags"] != 0
    ok = ~boundary
    mse = float(np.mean(d ** 2))
    rep = dict(max_abs=float(d[ok].max()) if ok.any() else 0.0,
               max_abs_all=float(d.max()),
               # pixels (boundary or not) off by more than the per-pixel bound
               over_tol_frac=float((d.max(-1) > TOL_MAX_ABS).mean()),
               psnr=float(10 * np.log10(1.0 / max(mse, 1e-30))),
               boundary_px=int(boundary.sum()), boundary_frac=float(boundary.mean()),
               covered_frac=float((ref["rgba"][..., 3] > 0).mean()),
               nonfinite=int((~np.isfinite(g)).sum()))
    return rep


def tile_lists_gpu(r, inst, gau):
    """{tile: int64 keys instance << 32 | gaussian} in GPU order."""
    rng = r.debug("tile_ranges").astype(np.int64)
    vals = r.debug("pair_splats").astype(np.int64)
    out = {}
    for t, (a, b) in enumerate(rng):
        if b > a:
            s = vals[a:b]
            out[t] = (inst[s] << 32) | gau[s]
    return out


def support_entries_per_row(os_, n_instances, W, H):
    """Per image row, the oracle's (pixel, splat) support-box entries: the
    widths of the clipped support boxes of every valid splat that covers the
    row (memory planning of banded full-frame renders)."""
    rows = np.zeros(H + 1, np.int64)
    for i in range(n_instances):
        p = oracle.project_instance(os_, i)
        g = np.nonzero(p["valid"])[0]
        if g.size == 0:
            continue
        u, v, r = p["uv"][g, 0], p["uv"][g, 1], p["radius"][g].astype(np.float64) + 1.0
        x0 = np.maximum(0, np.ceil(u - r - 0.5)); x1 = np.minimum(W - 1, np.floor(u + r - 0.5))
        y0 = np.maximum(0, np.ceil(v - r - 0.5)).astype(np.int64)
        y1 = np.minimum(H - 1, np.floor(v + r - 0.5)).astype(np.int64)
        ok = (x0 <= x1) & (y0 <= y1)
        w = (x1 - x0 + 1)[ok].astype(np.int64)
        np.add.at(rows, y0[ok], w)
        np.add.at(rows, y1[ok] + 1, -w)
    return np.cumsum(rows)[:H]


def render_banded(os_, eps, entries_per_row, budget=12_000_000):
    """oracle.render of the whole image in bands of rows, each holding at
    most about `budget` support-box entries; a single row over the budget
    is split into column ranges.  Stitched into one result."""
    W, H = os_.width, os_.height
    bands, y = [], 0
    while y < H:
        y1, acc = y, 0
        while y1 < H and (y1 == y or acc + entries_per_row[y1] <= budget):
            acc += int(entries_per_row[y1])
            y1 += 1
        parts = []
        nc = max(1, -(-acc // budget)) if y1 == y + 1 else 1
        for c in range(nc):
            x0, x1 = W * c // nc, W * (c + 1) // nc
            parts.append(oracle.render(os_, eps, lattice=(x0, y, 1, 1, x1 - x0, y1 - y)))
        bands.append({k: np.concatenate([p[k] for p in parts], 1) for k in parts[0]})
        y = y1
    return {k: np.concatenate([b_[k] for b_ in bands], 0) for k in bands[0]}


def compare_tile_lists(gl, ol, info, eps, W, H, tiles_x, tiles=None):
    """GPU tile lists `gl` against the oracle's `ol` (both {tile: keys in
    order}), over `tiles` (default: every tile of either).  A listed splat
    whose support-box edge lies within eps.px of a pixel centre, or whose
    3 sqrt(lambda) lies within eps.radius of an integer, is a boundary splat
    (it may be on one side only).  Pairs only the oracle lists must be
    unreachable (alpha < 1/255 over the tile's part of the box, FP64), and
    the common pairs must be in the same order except inside runs of
    near-equal depth.  Returns counts; asserts the rules."""
    n_pairs = n_dropped = perms = n_boundary = 0
    tiles = sorted(set(gl) | set(ol)) if tiles is None else tiles
    for t in tiles:
        G = gl.get(t, np.zeros(0, np.int64)).tolist()
        O = ol.get(t, np.zeros(0, np.int64)).tolist()
        n_pairs += len(G)
        sG, sO = set(G), set(O)

        def boundary(k):
            u, v, rr, rex = info[k][:4]
            e = np.array([u - rr - 0.5, u + rr - 0.5, v - rr - 0.5, v + rr - 0.5])
            return bool((np.abs(e - np.round(e)) < eps.px).any() or abs(rex - round(rex)) < eps.radius)

        extra = [k for k in sG - sO if not (k in info and boundary(k))]
        assert not extra, (t, extra[:5])
        missing = [k for k in sO - sG if not boundary(k)]
        n_boundary += len(sO ^ sG) - len(missing)
        if missing:
            a = np.array([info[k] for k in missing], np.float64)
            u, v, rr, A, B, C, o = a[:, 0], a[:, 1], a[:, 2], a[:, 4], a[:, 5], a[:, 6], a[:, 7]
            tx, ty = t % tiles_x, t // tiles_x
            x0 = np.maximum(tx * 16, np.maximum(0, np.ceil(u - rr - 0.5)))
            x1 = np.minimum(tx * 16 + 15, np.minimum(W - 1, np.floor(u + rr - 0.5)))
            y0 = np.maximum(ty * 16, np.maximum(0, np.ceil(v - rr - 0.5)))
            y1 = np.minimum(ty * 16 + 15, np.minimum(H - 1, np.floor(v + rr - 0.5)))
            f = rect_fmin(u, v, A, B, C, x0, x1, y0, y1)
            cut = 2 * np.log(255.0 * o)
            assert (f > cut - 2e-3).all(), (t, np.array(missing)[f <= cut - 2e-3][:5])
            n_dropped += len(missing)
        common = sG & sO
        Gc = [k for k in G if k in common]
        Oc = [k for k in O if k in common]
        if Gc != Oc:
            perms += 1
            d = np.array([info[k][8] for k in Gc])
            # the GPU order may differ only inside runs of near-equal depth
            assert (np.diff(d) >= -eps.depth_rel * np.maximum(1.0, d[1:]) * 4).all(), t
    return dict(pairs=n_pairs, dropped_unreachable=n_dropped, boundary_pairs=n_boundary, tiles_with_tie_perms=perms)
