"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI, read and
write workspace regions, and compare against the FP64 oracle.

Inputs always come from the seeded generators or from the oracle; nothing computed by the
CUDA path is ever fed to the oracle."""
from __future__ import annotations

import numpy as np
import torch

from oracle import projection as OP
from oracle import raster as R
from paper_2408_12894_gb300 import flod, synth

# tolerances (float32 path vs float64 oracle)
IMG_MAX_ABS = 2e-4      # per pixel and channel, on >= 99.9% of pixels
IMG_FRAC = 0.999
IMG_MEAN_ABS = 1e-5     # per channel
GRAD_REL = 1e-3         # ||g_gpu - g_ref|| / ||g_ref|| per parameter tensor, and per entry
GRAD_FLOOR = 1e-6       # elementwise: |d| <= GRAD_REL |g_ref| + GRAD_FLOOR max |g_ref|
DECISION_MARGIN = 2e-4  # relative distance of a blending decision to its threshold below
                        # which float32 and float64 may decide differently


def rasterizer(sets_np, cams, s_mins, view_sets=None, cfg=None, pair_capacity=None):
    sets = [flod.GaussianSet.from_numpy(g, s) for g, s in zip(sets_np, s_mins)]
    view_sets = view_sets if view_sets is not None else [0] * len(cams)
    views = [flod.view_struct(c, vs) for c, vs in zip(cams, view_sets)]
    return flod.Rasterizer(sets, views, cfg, pair_capacity)


def oracle_cfg(cfg) -> R.Config:
    return R.Config(tile_w=cfg.tile_w, tile_h=cfg.tile_h, dilation=float(cfg.dilation),
                    z_near=float(cfg.z_near), bg=tuple(float(x) for x in cfg.bg),
                    extent_rule=cfg.extent_rule)


def oracle_pre(g, s_min, cam, ocfg):
    with torch.no_grad():
        return R.preprocess(R.params(g), g["sh_degree"], s_min, cam, ocfg)


def units(rast, view: int, n: int) -> dict:
    """The preprocess outputs of the first n units of a view, as numpy arrays."""
    u0 = rast.unit_off[view]
    U = rast.layout.units
    out = {
        "xy": rast.region("xy", torch.float32, 2 * U).view(-1, 2)[u0:u0 + n],
        "depth": rast.region("depth", torch.float32, U)[u0:u0 + n],
        "conic_o": rast.region("conic_o", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n],
        "rgb": rast.region("rgb", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n],
        "radius": rast.region("radius", torch.float32, U)[u0:u0 + n],
        "ext": rast.region("ext", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n],
        "trec": rast.region("trec", torch.int32, 4 * U).view(-1, 4)[u0:u0 + n],
        "tiles_touched": rast.region("tiles_touched", torch.int32, U)[u0:u0 + n],
    }
    return {k: v.cpu().numpy() for k, v in out.items()}


def sorted_pairs(rast):
    """(keys uint64, vals uint32, ranges [tiles,2], pair_count, status) after bin_sort.

    The workspace keeps the 32-bit tile id of every sorted pair; the 64-bit sort key
    (tile << 32 | depth bits) is rebuilt from it and the depth of the pair's unit."""
    torch.cuda.synchronize()
    P = int(rast.pair_count.item())
    plan = rast.region("plan", torch.int32, 64).cpu().numpy()
    fin = int(plan[63])
    cap = rast.pair_capacity
    Pe = min(P, cap)
    tiles = rast.region("keys", torch.int32, cap, fin)[:Pe].cpu().numpy().view(np.uint32)
    vals = rast.region("vals", torch.int32, cap, fin)[:Pe].cpu().numpy().view(np.uint32)
    dbits = rast.region("depth", torch.float32, rast.layout.units).cpu().numpy().view(np.uint32)
    keys = (tiles.astype(np.uint64) << np.uint64(32)) | dbits[vals].astype(np.uint64)
    ranges = rast.region("ranges", torch.int32, 2 * rast.layout.tiles).view(-1, 2).cpu().numpy()
    status = flod.flod_read_status(rast.ws)
    return keys, vals, ranges.astype(np.int64), P, status


def image_compare(gpu_img: np.ndarray, ref_img: np.ndarray):
    """Returns (fraction of pixels within IMG_MAX_ABS, per-channel mean abs error)."""
    d = np.abs(gpu_img.astype(np.float64) - ref_img)
    per_pixel = d.max(axis=0)
    return float((per_pixel <= IMG_MAX_ABS).mean()), d.reshape(3, -1).mean(axis=1)


def assert_image_close(gpu_img, ref_img):
    frac, mean = image_compare(gpu_img, ref_img)
    assert frac >= IMG_FRAC, f"only {frac:.5f} of pixels within {IMG_MAX_ABS}"
    assert np.all(mean <= IMG_MEAN_ABS), f"mean abs error per channel {mean}"


def rect_boundary_distance(u, v, r):
    """FP64 distance of the four rectangle edges (u +- r - 0.5, v +- r - 0.5) to the nearest
    integer: the decisions a float32 pipeline may take differently."""
    u, v, r = (np.asarray(a, dtype=np.float64) for a in (u, v, r))
    ds = []
    for c in (u, v):
        for s in (-1.0, 1.0):
            x = c + s * r - 0.5
            ds.append(np.abs(x - np.round(x)))
    return np.minimum.reduce(ds)


def unit_tile_sets_f32(u, v, r, ext, valid, cam, ocfg):
    """tiles_touched, the tile rectangle and the row segments of float32 units, decided in
    float32 with the kernels' operations (rules 0 and 1: the square of radius r; rule 2: the
    rows of the support ellipse ext)."""
    W, H = cam["width"], cam["height"]
    if ocfg.extent_rule == 2:
        ext = np.asarray(ext, dtype=np.float32)
        px = OP.pixel_rect_xy(u, v, ext[:, 2], ext[:, 3], W, H, np.float32)
        segs, touched = OP.ellipse_segments(u, v, ext, px, ocfg.tile_w, ocfg.tile_h, valid,
                                            np.float32)
        tr = OP.tile_rect(px, ocfg.tile_w, ocfg.tile_h, valid & (touched > 0))
    else:
        px = OP.pixel_rect_f32(u, v, r, W, H)
        tr = OP.tile_rect(px, ocfg.tile_w, ocfg.tile_h, valid)
        touched = tr[4]
        segs = OP.rect_segments(tr[:4], touched)
    return touched, tr[:4], segs


def tile_records(f, ocfg):
    """The per-unit tile record the emission reads (uint32 [n, 4]), from a unit dict with
    "tile_rect", "segments" and "valid": x = tx0 | ty0 << 16, y = rows | mode << 16; mode 0
    holds up to 4 rows of (column offset, count) bytes in z, w; mode 1 (rectangle rules) the
    per-row count in z; mode 2 (more rows, or a byte overflows) is recomputed by the kernel."""
    tx0, tx1, ty0, ty1 = (np.asarray(a, dtype=np.int64) for a in f["tile_rect"])
    n = tx0.size
    valid = np.asarray(f["valid"], dtype=bool)
    rec = np.zeros((n, 4), dtype=np.uint32)
    rows = np.where(valid, ty1 - ty0 + 1, 0)
    rec[:, 0] = np.where(valid, tx0 | (ty0 << 16), 0)
    if ocfg.extent_rule != 2:
        rec[:, 1] = np.where(valid, rows | (1 << 16), 0)
        rec[:, 2] = np.where(valid, tx1 - tx0 + 1, 0)
        return rec
    mode = np.where(rows > 4, 2, 0)
    su, sy, sx0, sx1 = (np.asarray(a, dtype=np.int64) for a in f["segments"])
    keep = valid[su]
    su, sy, sx0, sx1 = su[keep], sy[keep], sx0[keep], sx1[keep]
    r = sy - ty0[su]
    off, cnt = sx0 - tx0[su], sx1 - sx0 + 1
    first = r < 4
    over = np.zeros(n, bool)
    np.logical_or.at(over, su[first], (off[first] > 255) | (cnt[first] > 255))
    mode = np.where(over, 2, mode)
    h = (off & 0xff) | ((cnt & 0xff) << 8)
    for rr in range(4):
        sel = first & (r == rr)
        word, shift = 2 + rr // 2, 16 * (rr % 2)
        np.bitwise_or.at(rec[:, word], su[sel], (h[sel] << shift).astype(np.uint32))
    rec[:, 1] = np.where(valid, rows | (mode << 16), 0)
    return rec


def oracle_units_f32(pre, cam, ocfg):
    """The oracle's FP64 preprocess rounded to float32, with the tile sets decided in float32
    by the same rule (so an integer stage fed with it has one exact answer)."""
    valid = pre["valid"].numpy()
    u = pre["mean2d"][:, 0].detach().numpy().astype(np.float32)
    v = pre["mean2d"][:, 1].detach().numpy().astype(np.float32)
    r = pre["radius"].numpy().astype(np.float32)
    ext = pre["ext"].numpy().astype(np.float32)
    u, v, r = (np.where(valid, a, np.float32(0)) for a in (u, v, r))
    ext = np.where(valid[:, None], ext, np.float32(0))
    touched, tr, segs = unit_tile_sets_f32(u, v, r, ext, valid, cam, ocfg)
    return {"u": u, "v": v, "r": r, "ext": ext,
            "depth": pre["depth"].detach().numpy().astype(np.float32),
            "conic": pre["conic"].detach().numpy().astype(np.float32),
            "opacity": pre["opacity"].detach().numpy().astype(np.float32),
            "rgb": pre["rgb"].detach().numpy().astype(np.float32),
            "valid": valid & (touched > 0), "tile_rect": tr, "segments": segs,
            "tiles_touched": touched}


def random_units_f32(rng, n, cam, ocfg, r_scale=4.0, aniso=20.0, depth=None):
    """Synthetic float32 units with random support ellipses (any orientation, anisotropy up to
    ``aniso``), partly off-screen, and their float32 tile sets."""
    W, H = cam["width"], cam["height"]
    u = rng.uniform(-50, W + 50, n).astype(np.float32)
    v = rng.uniform(-50, H + 50, n).astype(np.float32)
    th = rng.uniform(0, np.pi, n)
    s1 = rng.gamma(2.0, r_scale, n) + 0.3
    s2 = s1 / np.exp(rng.uniform(0, np.log(aniso), n)) + 0.3
    c, sn = np.cos(th), np.sin(th)
    A = c * c * s1 * s1 + sn * sn * s2 * s2
    B = c * sn * (s1 * s1 - s2 * s2)
    C = sn * sn * s1 * s1 + c * c * s2 * s2
    ext = np.stack([B / C, np.sqrt(A * C - B * B) / C, np.sqrt(A), np.sqrt(C)], 1)
    ext = ext.astype(np.float32)
    r = np.sqrt(0.5 * (A + C) + np.sqrt(0.25 * (A - C) ** 2 + B * B)).astype(np.float32)
    valid = rng.random(n) > 0.05
    touched, tr, segs = unit_tile_sets_f32(u, v, r, ext, valid, cam, ocfg)
    d = rng.uniform(20, 60, n).astype(np.float32) if depth is None else depth
    return {"u": u, "v": v, "r": r, "ext": ext, "depth": d,
            "valid": valid & (touched > 0), "tile_rect": tr, "segments": segs,
            "tiles_touched": touched}


def inject_units(rast, view: int, f: dict):
    """Write oracle-made per-unit values into the workspace of a view."""
    n = f["u"].shape[0]
    u0 = rast.unit_off[view]
    U = rast.layout.units
    dev = rast.ws.device
    xy = np.stack([f["u"], f["v"]], 1).astype(np.float32)
    rast.region("xy", torch.float32, 2 * U).view(-1, 2)[u0:u0 + n] = torch.as_tensor(xy, device=dev)
    rast.region("depth", torch.float32, U)[u0:u0 + n] = torch.as_tensor(f["depth"], device=dev)
    rast.region("radius", torch.float32, U)[u0:u0 + n] = torch.as_tensor(f["r"], device=dev)
    rast.region("ext", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n] = \
        torch.as_tensor(np.ascontiguousarray(f["ext"], dtype=np.float32), device=dev)
    rec = tile_records(f, oracle_cfg(rast.cfg)).view(np.int32)
    rast.region("trec", torch.int32, 4 * U).view(-1, 4)[u0:u0 + n] = torch.as_tensor(rec, device=dev)
    tt = np.where(f["valid"], f["tiles_touched"], 0).astype(np.int32)
    rast.region("tiles_touched", torch.int32, U)[u0:u0 + n] = torch.as_tensor(tt, device=dev)
    if "conic" in f:
        co = np.concatenate([f["conic"], f["opacity"][:, None]], 1).astype(np.float32)
        rast.region("conic_o", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n] = torch.as_tensor(co, device=dev)
        rgb = np.concatenate([f["rgb"], np.zeros((n, 1), np.float32)], 1)
        rast.region("rgb", torch.float32, 4 * U).view(-1, 4)[u0:u0 + n] = torch.as_tensor(rgb, device=dev)


def clear_units(rast):
    U = rast.layout.units
    rast.region("tiles_touched", torch.int32, U).zero_()


def assert_grad_close(got: dict, ref: dict, what: str = "", floor_abs: float = 0.0,
                      mag: dict | None = None):
    """Both bars of the gradient parity: per parameter tensor, relative L2 error <= GRAD_REL,
    and per entry |g - g_ref| <= GRAD_REL |g_ref| + GRAD_FLOOR max|g_ref| + floor_abs (max over
    the compared entries of that tensor; floor_abs is 0 except where a test derives one).
    mag (optional, same keys and shapes): for a gradient that is a sum of separately computed
    terms (views), the sum of the terms' magnitudes, which the per-entry relative bar is then
    taken of (float32 rounds the terms, not their possibly cancelling sum)."""
    for k in ref:
        a = np.asarray(got[k], dtype=np.float64).reshape(-1)
        b = np.asarray(ref[k], dtype=np.float64).reshape(-1)
        scale = np.abs(b) if mag is None else np.maximum(np.abs(b), np.asarray(mag[k], np.float64).reshape(-1))
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.all(a == 0), f"{what} {k}: nonzero gradient where the oracle's is zero"
            continue
        rel = np.linalg.norm(a - b) / nb
        assert rel <= GRAD_REL, f"{what} {k}: relative L2 error {rel:.2e}"
        bound = GRAD_REL * scale + GRAD_FLOOR * np.abs(b).max() + floor_abs
        bad = np.nonzero(np.abs(a - b) > bound)[0]
        assert bad.size == 0, (f"{what} {k}: {bad.size} of {b.size} entries off, worst "
                               f"|d|={np.abs(a - b)[bad].max():.3e} at |g_ref|={np.abs(b)[bad[0]]:.3e}")


def blend_decision_margin(pix_xy, mean2d, conic, opacity):
    """FP64 relative distance of every discrete blending decision of each pixel to its
    threshold: alpha against 1/255 for each Gaussian up to the one that stops the pixel, and
    T (1 - alpha) against 1e-4 for each blended one. A pixel whose smallest margin is below
    DECISION_MARGIN may blend another set of Gaussians in float32; elsewhere n_contrib has
    one right answer. Inputs are torch float64 (pixel centres [P,2], the tile's Gaussians
    in list order)."""
    with torch.no_grad():
        a_raw = R.alpha_raw(pix_xy, mean2d, conic, opacity).numpy()
    if a_raw.shape[1] == 0:
        return np.full(a_raw.shape[0], np.inf)
    a = np.minimum(a_raw, R.ALPHA_MAX)
    kept = a >= R.ALPHA_MIN
    m_skip = np.where(a_raw < R.ALPHA_MAX, np.abs(a_raw / R.ALPHA_MIN - 1.0), np.inf)
    t_after = np.cumprod(1.0 - np.where(kept, a, 0.0), axis=1)
    m_stop = np.where(kept, np.abs(t_after / R.T_MIN - 1.0), np.inf)
    live = t_after >= R.T_MIN
    K = a.shape[1]
    stop = np.where(live.all(axis=1), K - 1, np.argmin(live, axis=1))
    upto = np.arange(K)[None, :] <= stop[:, None]
    m = np.where(upto, np.minimum(m_skip, m_stop), np.inf)
    return m.min(axis=1)


def tile_sample(ranges_tile, tiles_x, tiles_y, n, rng):
    """About n tiles of one view: stratified over the pair-count distribution (empty to
    heaviest) plus the four corners and a ragged last row / column tile."""
    counts = ranges_tile[:, 1] - ranges_tile[:, 0]
    order = np.argsort(counts, kind="stable")
    k = max(n - 6, 1)
    picks = set(int(order[int(q)]) for q in np.linspace(0, order.size - 1, k))
    picks |= {0, tiles_x - 1, tiles_x * (tiles_y - 1), tiles_x * tiles_y - 1,
              (tiles_y - 1) * tiles_x + tiles_x // 2, (tiles_y // 2) * tiles_x + tiles_x - 1}
    extra = rng.choice(tiles_x * tiles_y, size=2, replace=False)
    picks |= set(int(t) for t in extra)
    return sorted(picks)


def blended_gaussians(lists, ref_tiles):
    """Candidates for sampled-gradient checks: the Gaussians of the oracle's tile lists, in
    the sampled tiles it rendered, up to each tile's last blended position. A Gaussian behind
    every pixel's stop (or culled) has an exactly zero gradient, and a sample of such
    Gaussians would compare zeros with zeros."""
    _, vals, ranges, _, _ = lists
    out = set()
    for t, (_, _, last) in ref_tiles.items():
        s = int(ranges[t][0])
        out.update(int(x) for x in vals[s:s + int(np.max(last))])
    return np.array(sorted(out), dtype=np.int64)


def assert_nonvacuous(ref, what="", min_frac=0.75):
    """At least min_frac of the sampled Gaussians have a nonzero reference gradient."""
    nz = None
    for v in ref.values():
        a = np.abs(np.asarray(v)).reshape(np.asarray(v).shape[0], -1).max(axis=1) > 0
        nz = a if nz is None else (nz | a)
    assert nz.mean() >= min_frac, f"{what}: only {int(nz.sum())} of {nz.size} sampled gradients are nonzero"


def compare_tiles(img, T, nc, ref_tiles, pre, lists, cam, ocfg, gpu_lists=None):
    """GPU outputs ([3,H,W], [H,W], [H,W] numpy) against the oracle's render of the sampled
    tiles (R.render_tiles). n_contrib is a 1-based position in a tile's list: with
    ``gpu_lists`` = (the GPU's sorted Gaussian indices, its [tiles, 2] ranges) of this view,
    each side's position is turned into the Gaussian it names and those are compared (the two
    lists may differ by Gaussians at the edge of their tile sets, which no pixel blends);
    without it the lists are the same and positions are compared. Returns (per-pixel max abs
    error over channels, per-channel abs errors, T abs errors, last blended Gaussian equal
    where the decisions are unambiguous, fraction of pixels with an ambiguous decision)."""
    keys, vals, ranges, tx, ty = lists
    pix_err, ch_err, t_err, nc_ok, amb = [], [], [], [], []
    for t, (col, tf, last) in ref_tiles.items():
        x0, y0, x1, y1 = R.tile_pixels(t, tx, cam, ocfg)
        d = np.abs(img[:, y0:y1, x0:x1].astype(np.float64) - col).reshape(3, -1)
        pix_err.append(d.max(axis=0))
        ch_err.append(d)
        t_err.append(np.abs(T[y0:y1, x0:x1].astype(np.float64) - tf).reshape(-1))
        s, e = ranges[t]
        g = torch.as_tensor(vals[s:e].astype(np.int64))
        gx, gy = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1))
        pix = torch.as_tensor(np.stack([gx.ravel() + 0.5, gy.ravel() + 0.5], 1).astype(np.float64))
        m = blend_decision_margin(pix, pre["mean2d"].detach()[g], pre["conic"].detach()[g],
                                  pre["opacity"].detach()[g])
        clear = m > DECISION_MARGIN
        got = nc[y0:y1, x0:x1].reshape(-1).astype(np.int64)
        want = last.reshape(-1).astype(np.int64)
        if gpu_lists is not None:
            gv, gr = gpu_lists
            gs, ge = (int(x) for x in gr[t])
            got = np.where(got > 0, np.asarray(gv[gs:ge], np.int64)[np.maximum(got - 1, 0)]
                           if ge > gs else -1, -1)
            want = np.where(want > 0, vals[s:e].astype(np.int64)[np.maximum(want - 1, 0)]
                            if e > s else -1, -1)
        nc_ok.append(np.where(clear, got == want, True))
        amb.append(~clear)
    return (np.concatenate(pix_err), np.concatenate(ch_err, axis=1), np.concatenate(t_err),
            np.concatenate(nc_ok), float(np.concatenate(amb).mean()))


def assert_tiles_close(img, T, nc, ref_tiles, pre, lists, cam, ocfg, what="", gpu_lists=None):
    """The image bar on the sampled tiles' pixels (>= 99.9% within 2e-4, mean abs <= 1e-5
    per channel), T within 2e-4 on >= 99.9% of them, and the last blended Gaussian equal
    wherever the blending decisions are unambiguous (ambiguous pixels: under 5%)."""
    pe, ce, te, ncok, amb = compare_tiles(img, T, nc, ref_tiles, pre, lists, cam, ocfg, gpu_lists)
    frac = float((pe <= IMG_MAX_ABS).mean())
    assert frac >= IMG_FRAC, f"{what}: only {frac:.5f} of {pe.size} pixels within {IMG_MAX_ABS}"
    mean = ce.mean(axis=1)
    assert np.all(mean <= IMG_MEAN_ABS), f"{what}: mean abs error per channel {mean}"
    tfrac = float((te <= IMG_MAX_ABS).mean())
    assert tfrac >= IMG_FRAC, f"{what}: T within {IMG_MAX_ABS} on only {tfrac:.5f}"
    assert amb < 0.05, f"{what}: {amb:.4f} of pixels have an ambiguous blending decision"
    assert ncok.all(), f"{what}: last blended Gaussian differs on {int((~ncok).sum())} pixels"
    return pe.size


def gpu_view_lists(rast, view: int):
    """The GPU's sorted Gaussian indices of one view (unit offset of the view removed; a
    selective view's indices are positions in its selection list) and the view's [tiles, 2]
    ranges into them. Only the view's slice of the pair list is read back (a view's pairs are
    contiguous: tile ids are global, views in order)."""
    torch.cuda.synchronize()
    fin = int(rast.region("plan", torch.int32, 64)[63].item())
    t0, t1 = rast.tile_off[view], rast.tile_off[view + 1]
    rg = rast.region("ranges", torch.int32, 2 * rast.layout.tiles).view(-1, 2)[t0:t1]
    rg = rg.cpu().numpy().astype(np.int64)
    full = rg[:, 1] > rg[:, 0]
    lo = int(rg[full, 0].min()) if full.any() else 0
    hi = int(rg[full, 1].max()) if full.any() else 0
    vals = rast.region("vals", torch.int32, rast.pair_capacity, fin)[lo:hi]
    vals = vals.cpu().numpy().astype(np.int64)
    rg = np.where(full[:, None], rg - lo, 0)
    return vals - rast.unit_off[view], rg
