"""Renderer for seeded synthetic orthogonal scan pairs (see package docstring)."""
import math

import numpy as np
from scipy.special import ndtr

# Workload presets.  Sizes, layer/slab/saccade counts and drift follow the
# configurations the benchmark and tests use; seed = 1000 + preset number.
CONFIGS = {
    # plain method, small: single level
    "c1": dict(w=64, h=64, d=64, n_layers=8, n_slabs=2, n_saccades=2, max_saccade=5.0,
               drift_sigma=0.02, levels=1, seed=1001),
    # plain method, clinical size: 3-level pyramid
    "c2": dict(w=300, h=300, d=512, n_layers=12, n_slabs=3, n_saccades=6, max_saccade=15.0,
               drift_sigma=0.03, levels=3, seed=1002),
    # precision: wide field
    "c3": dict(w=600, h=600, d=800, n_layers=12, n_slabs=3, n_saccades=10, max_saccade=25.0,
               drift_sigma=0.03, levels=3, seed=1003),
    # differentiation
    "c4": dict(w=128, h=128, d=256, n_layers=8, n_slabs=2, n_saccades=3, max_saccade=8.0,
               drift_sigma=0.03, levels=1, seed=1004),
}

FLYBACK = 0.25        # flyback slots per B-scan, as a fraction of the A-scans per B-scan
SCAN_SECONDS = 3.9    # acquisition time of one volume, kept constant across sizes
AXIAL_AMP = 2.0       # px, 1 Hz axial sinusoid
AXIAL_HZ = 1.0
BUMP_HEIGHT = 6.0     # px, drusen-like elevation of the deepest surfaces
ANGIO_OVERSAMPLE = 4  # vessel map resolution per pixel
ANGIO_PAD = 64        # px of vessel map around the grid


# ------------------------------------------------------------------ scan pattern
def slots(w, h):
    """(n_fast_x, flyback) slot geometry: X-fast rows of w + f slots, Y-fast columns of h + f."""
    return int(round(FLYBACK * w)), int(round(FLYBACK * h))


def time_maps(w, h):
    """Sampling-time maps in slot units: X-fast raster along i, Y-fast along j."""
    fx, fy = slots(w, h)
    j, i = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    tx = j * (w + fx) + i
    ty = i * (h + fy) + j
    return tx, ty


# ------------------------------------------------------------------ motion
def _motion(rng, n_slots, drift_sigma, n_saccades, max_saccade, smooth_amp=0.0):
    """Eye position m(s) per slot: drift + saccades (x, y) + axial sinusoid (z),
    plus, with smooth_amp > 0, slow transverse sinusoids of that amplitude."""
    m = np.cumsum(rng.normal(0.0, drift_sigma, size=(n_slots, 3)), axis=0)
    sac = np.sort(rng.integers(1, n_slots, size=n_saccades))
    cur = np.zeros(2)
    for s in sac:
        ang = rng.uniform(0.0, 2.0 * math.pi)
        mag = rng.uniform(0.3, 1.0) * max_saccade
        jump = mag * np.array([math.cos(ang), math.sin(ang)])
        if np.hypot(*(cur + jump)) > max_saccade:  # keep fixation bounded
            jump = -jump
        cur = cur + jump
        m[s:, :2] += jump
    seconds = np.arange(n_slots) * (SCAN_SECONDS / n_slots)
    m[:, 2] += AXIAL_AMP * np.sin(2.0 * math.pi * AXIAL_HZ * seconds + rng.uniform(0, 2 * math.pi))
    if smooth_amp > 0.0:
        for c in range(2):
            hz, ph = rng.uniform(0.2, 0.6), rng.uniform(0, 2 * math.pi)
            m[:, c] += smooth_amp * np.sin(2.0 * math.pi * hz * seconds + ph)
    return m, sac


# ------------------------------------------------------------------ retina
class _Retina:
    def __init__(self, rng, w, h, d, n_layers):
        self.n = n_layers
        self.top = d * rng.uniform(0.18, 0.26)
        thick = rng.uniform(0.5, 1.5, size=n_layers)
        self.offsets = np.concatenate([[0.0], np.cumsum(thick * (0.45 * d / thick.sum()))])
        amp = rng.uniform(0.15, 0.9, size=n_layers)
        amp[-1] = 1.0  # bright RPE-like band
        self.levels = np.concatenate([[0.03], amp, [0.25]])  # above, bands, below
        self.cx, self.cy = w * rng.uniform(0.4, 0.6), h * rng.uniform(0.4, 0.6)
        self.r2 = (0.5 * w) ** 2 + (0.5 * h) ** 2
        self.curv = d * rng.uniform(0.05, 0.1)
        self.bx, self.by = w * rng.uniform(0.3, 0.7), h * rng.uniform(0.3, 0.7)
        self.bsig = 0.08 * max(w, h)
        self.sigma = 1.2

    def surfaces(self, x, y):
        """Surface depths [..., n+1] at transverse positions x, y."""
        bowl = -self.curv * ((x - self.cx) ** 2 + (y - self.cy) ** 2) / self.r2
        bump = BUMP_HEIGHT * np.exp(-((x - self.bx) ** 2 + (y - self.by) ** 2) / (2 * self.bsig ** 2))
        s = self.top + self.offsets + bowl[..., None]
        s[..., -2:] -= bump[..., None]
        return s

    def render(self, x, y, z0, d):
        """Intensity [..., d] of A-scans at (x, y) sampled at depths k + z0."""
        surf = self.surfaces(x, y).astype(np.float32)
        z = np.arange(d, dtype=np.float32) + z0[..., None].astype(np.float32)
        out = np.full(z.shape, self.levels[0], dtype=np.float32)
        steps = np.diff(self.levels).astype(np.float32)
        inv = np.float32(1.0 / self.sigma)
        for l in range(self.n + 1):
            out += steps[l] * ndtr((z - surf[..., l:l + 1]) * inv).astype(np.float32)
        return out


# ------------------------------------------------------------------ vessels
def _vessel_segments(rng, w, h):
    segs = []
    n_roots = 3 + max(w, h) // 100
    for _ in range(n_roots):
        stack = [(rng.uniform(0, w), rng.uniform(0, h), rng.uniform(0, 2 * math.pi), 3.0, 0)]
        while stack:
            x, y, ang, width, depth = stack.pop()
            length = rng.uniform(0.08, 0.25) * max(w, h)
            for _p in range(4):
                ang += rng.normal(0.0, 0.25)
                x1, y1 = x + math.cos(ang) * length / 4, y + math.sin(ang) * length / 4
                segs.append((x, y, x1, y1, width))
                x, y = x1, y1
            if depth < 4 and width > 1.0:
                for sgn in (-1.0, 1.0):
                    stack.append((x, y, ang + sgn * rng.uniform(0.3, 0.9), max(1.0, 0.75 * width),
                                  depth + 1))
    return segs


def _rasterise(segs, w, h):
    """Vessel map on a grid oversampled ANGIO_OVERSAMPLE x, padded by ANGIO_PAD px."""
    o, pad = ANGIO_OVERSAMPLE, ANGIO_PAD
    W, H = (w + 2 * pad) * o, (h + 2 * pad) * o
    img = np.zeros((H, W), dtype=np.float32)
    for (x0, y0, x1, y1, width) in segs:
        r = 1.5 * width + 1
        xa, xb = int(max((min(x0, x1) - r + pad) * o, 0)), int(min((max(x0, x1) + r + pad) * o + 1, W))
        ya, yb = int(max((min(y0, y1) - r + pad) * o, 0)), int(min((max(y0, y1) + r + pad) * o + 1, H))
        if xa >= xb or ya >= yb:
            continue
        gx = np.arange(xa, xb, dtype=np.float32) / o - pad
        gy = np.arange(ya, yb, dtype=np.float32) / o - pad
        px, py = np.meshgrid(gx, gy)
        dx, dy = x1 - x0, y1 - y0
        ll = dx * dx + dy * dy
        t = np.clip(((px - x0) * dx + (py - y0) * dy) / max(ll, 1e-9), 0.0, 1.0)
        dist2 = (px - x0 - t * dx) ** 2 + (py - y0 - t * dy) ** 2
        val = np.exp(-dist2 / (2.0 * (0.5 * width) ** 2)).astype(np.float32)
        np.maximum(img[ya:yb, xa:xb], val, out=img[ya:yb, xa:xb])
    return img


def _sample_map(img, x, y):
    """Bilinear sample of a rasterised map at continuous pixel positions (x, y)."""
    o, pad = ANGIO_OVERSAMPLE, ANGIO_PAD
    H, W = img.shape
    u = np.clip((x + pad) * o, 0, W - 1.001)
    v = np.clip((y + pad) * o, 0, H - 1.001)
    u0, v0 = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
    fu, fv = (u - u0).astype(np.float32), (v - v0).astype(np.float32)
    return ((1 - fu) * (1 - fv) * img[v0, u0] + fu * (1 - fv) * img[v0, u0 + 1] +
            (1 - fu) * fv * img[v0 + 1, u0] + fu * fv * img[v0 + 1, u0 + 1])


def _sample_grid(img, u, v):
    """Bilinear sample of a texture given at integer positions, at continuous (u, v):
    the texture moves with the eye as a continuous function of position."""
    H, W = img.shape
    u = np.clip(u, 0, W - 1.001)
    v = np.clip(v, 0, H - 1.001)
    u0, v0 = np.floor(u).astype(np.int64), np.floor(v).astype(np.int64)
    fu, fv = (u - u0).astype(np.float32), (v - v0).astype(np.float32)
    return ((1 - fu) * (1 - fv) * img[v0, u0] + fu * (1 - fv) * img[v0, u0 + 1] +
            (1 - fu) * fv * img[v0 + 1, u0] + fu * fv * img[v0 + 1, u0 + 1])


# ------------------------------------------------------------------ pair
def _interp_motion(m, s):
    """Motion at continuous slot positions s (linear, clamped)."""
    n = m.shape[0]
    s = np.clip(s, 0.0, n - 1.0)
    s0 = np.minimum(np.floor(s).astype(np.int64), n - 2) if n > 1 else np.zeros_like(s, dtype=np.int64)
    f = (s - s0)[..., None]
    return (1 - f) * m[s0] + f * m[np.minimum(s0 + 1, n - 1)]


def _render_torch(retina, x, y, z0, d, speckle, gen, device):
    """The retina intensity (and speckle) of A-scans at (x, y) on a torch device."""
    import torch
    surf = torch.from_numpy(retina.surfaces(x, y).astype(np.float32)).to(device)
    z = torch.arange(d, dtype=torch.float32, device=device) + torch.from_numpy(
        np.asarray(z0, dtype=np.float32)).to(device)[..., None]
    out = torch.full(z.shape, float(retina.levels[0]), dtype=torch.float32, device=device)
    steps = np.diff(retina.levels)
    for l in range(retina.n + 1):
        out += float(steps[l]) * torch.special.ndtr((z - surf[..., l:l + 1]) / retina.sigma)
    if speckle:
        u = torch.rand(out.shape, generator=gen, device=device, dtype=torch.float32).clamp_min_(1e-12)
        out *= math.sqrt(2.0 / math.pi) * torch.sqrt(-2.0 * torch.log(u))  # unit-mean Rayleigh
    return out


def make_pair(w, h, d, n_layers=8, n_slabs=2, n_saccades=2, max_saccade=5.0, drift_sigma=0.02,
              seed=0, speckle=True, row_chunk=16, device=None, smooth_amp=0.0, angio_noise=True, **_unused):
    """Render one orthogonal scan pair.

    Returns a dict with float32 ``sx, sy [h][w][d]``, ``ax, ay [h][w]``,
    ``vx [h]``, ``vy [w]``, float64 ``tx, ty [h][w]`` and the motion
    (``mx, my`` per slot, [n][3]) with the saccade slots.  With ``device``
    (a torch device) the volumes are rendered there and returned as torch
    tensors (same structure and parameters; speckle from torch's generator),
    which is much faster for large pairs.
    """
    rng = np.random.default_rng(seed)
    retina = _Retina(rng, w, h, d, n_layers)
    fx, fy = slots(w, h)
    nx, ny = h * (w + fx), w * (h + fy)
    mx, sacx = _motion(rng, nx, drift_sigma, n_saccades, max_saccade, smooth_amp)
    my, sacy = _motion(rng, ny, drift_sigma, n_saccades, max_saccade, smooth_amp)
    tx, ty = time_maps(w, h)

    slab_maps = [_rasterise(_vessel_segments(rng, w, h), w, h) for _ in range(n_slabs)]
    slab_frac = rng.uniform(0.04, 0.1, size=n_slabs)
    angio_bg = rng.uniform(0.0, 1.0, size=(h + 2 * ANGIO_PAD, w + 2 * ANGIO_PAD)).astype(np.float32)

    def angio_at(x, y):
        a = np.zeros(x.shape, dtype=np.float32)
        for frac, mp in zip(slab_frac, slab_maps):
            a += np.float32(frac) * _sample_map(mp, x, y)
        return a / np.float32(slab_frac.sum())  # depth mean over the vessel slabs

    out = {}
    for name, m, tmap, sac, slow_len in (("x", mx, tx, sacx, h), ("y", my, ty, sacy, w)):
        srng = np.random.default_rng(seed * 7919 + (1 if name == "x" else 2))
        if device is not None:
            import torch
            gen = torch.Generator(device=device)
            gen.manual_seed(seed * 7919 + (1 if name == "x" else 2))
            s = tmap.astype(np.int64)
            mv = m[s]
            jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
            vol = _render_torch(retina, ii + mv[..., 0], jj + mv[..., 1], mv[..., 2], d, speckle, gen, device)
        else:
            vol = np.empty((h, w, d), dtype=np.float32)
        for j0 in range(0, h if device is None else 0, row_chunk):
            j1 = min(h, j0 + row_chunk)
            s = tmap[j0:j1].astype(np.int64)
            mv = m[s]
            jj, ii = np.meshgrid(np.arange(j0, j1), np.arange(w), indexing="ij")
            blk = retina.render(ii + mv[..., 0], jj + mv[..., 1], mv[..., 2], d)
            if speckle:
                blk *= srng.rayleigh(math.sqrt(2.0 / math.pi), size=blk.shape).astype(np.float32)
            vol[j0:j1] = blk
        s = tmap.astype(np.int64)
        jj, ii = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
        a = angio_at(ii + m[s, 0], jj + m[s, 1])
        noise = srng.normal(0.0, 0.01, size=a.shape).astype(np.float32)
        if angio_noise:
            a += np.float32(0.02) * _sample_grid(angio_bg, ii + m[s, 0] + ANGIO_PAD, jj + m[s, 1] + ANGIO_PAD)
            a += noise
        # saccades: B-scans within 2 of a jump are saturated and invalid (Sec. 2.2)
        valid = np.ones(slow_len, dtype=np.float32)
        fast = w + fx if name == "x" else h + fy
        for sl in sac:
            b = int(sl // fast)
            valid[max(0, b - 2):min(slow_len, b + 3)] = 0.0
        bad = np.where(valid == 0)[0]
        if name == "x":
            a[bad, :] = 1.0
        else:
            a[:, bad] = 1.0
        # nearest valid B-scan replaces an invalid one (Sec. 2.3, last step)
        good = np.where(valid > 0)[0]
        if good.size:
            for b in bad:
                nb = good[np.argmin(np.abs(good - b))]
                if name == "x":
                    a[b, :] = a[nb, :]
                else:
                    a[:, b] = a[:, nb]
        out["s" + name] = vol
        out["a" + name] = np.ascontiguousarray(a, dtype=np.float32)
        out["v" + name] = valid
        out["t" + name] = tmap
        out["m" + name] = m
        out["sac" + name] = sac
    return out


def make_config(name, **over):
    """Render a named preset (``c1`` ... ``c4``); keyword overrides win."""
    cfg = dict(CONFIGS[name])
    cfg.update(over)
    return make_pair(**cfg), cfg


def true_displacement(pair, w, h, iters=60):
    """Ground-truth displacement fields [2][3][h][w] and a validity mask [2][h][w].

    Solves p + d + m(t(p + d)) = p + c by damped fixed-point iteration, with the
    slot map extended linearly between A-scans; c makes the total displacement
    zero per component.  A-scans near a saccade are masked out (the solution
    there is not unique): the B-scans within 2 of the saccade, and, in the
    corrected frame, the band of slow-axis positions between where the
    saccade's B-scan lands before and after the jump (the gap or the overlap
    the jump leaves), widened by 2.5 B-scans on both sides.
    """
    fx, fy = slots(w, h)
    jj, ii = np.meshgrid(np.arange(h, dtype=np.float64), np.arange(w, dtype=np.float64), indexing="ij")
    disp = np.zeros((2, 3, h, w))
    mask = np.ones((2, h, w), dtype=bool)
    c = np.zeros(3)
    for _outer in range(4):
        for V, (m, sac) in enumerate(((pair["mx"], pair["sacx"]), (pair["my"], pair["sacy"]))):
            d = disp[V]
            for _ in range(iters):
                x, y = ii + d[0], jj + d[1]
                s = y * (w + fx) + x if V == 0 else x * (h + fy) + y
                mv = _interp_motion(m, s)
                new = c[:, None, None] - np.moveaxis(mv, -1, 0)
                d = 0.5 * d + 0.5 * new
            disp[V] = d
            fast = w + fx if V == 0 else h + fy
            for sl in sac:
                b = int(sl // fast)
                if V == 0:
                    mask[V, max(0, b - 2):b + 3, :] = False
                else:
                    mask[V, :, max(0, b - 2):b + 3] = False
        c = c - disp.mean(axis=(0, 2, 3))
    # the gap / overlap band of each saccade in the corrected frame: acquired
    # slow position b shows the object at b + m_slow - c_slow
    for V, (m, sac) in enumerate(((pair["mx"], pair["sacx"]), (pair["my"], pair["sacy"]))):
        fast = w + fx if V == 0 else h + fy
        slow = 1 if V == 0 else 0
        pos = jj if V == 0 else ii
        for sl in sac:
            b = sl / fast
            lo = b + min(m[sl - 1, slow], m[sl, slow]) - c[slow] - 2.5
            hi = b + max(m[sl - 1, slow], m[sl, slow]) - c[slow] + 2.5
            mask[V] &= ~((pos >= lo) & (pos <= hi))
    return disp, mask


INPUT_KEYS = ("sx", "sy", "ax", "ay", "vx", "vy", "tx", "ty")


def fingerprint(pair):
    """Per input array of a pair: its float64 sum and sum of squares.

    Equal renderings on two platforms may differ in the last bits of some
    voxels (their numpy builds round transcendental functions differently),
    so stored results are matched to their inputs by these sums to a relative
    tolerance rather than by a checksum of the bytes."""
    out = {}
    for k in INPUT_KEYS:
        a = pair.get(k)
        if a is None:
            continue
        a = np.asarray(a, dtype=np.float64)
        out[k] = [float(a.sum()), float((a * a).sum())]
    return out


def fingerprints_match(a, b, rel=3e-7):
    """True when two fingerprints name the same arrays with sums equal to
    ``rel`` relative.  Last-bit differences of a float32 rendering move a sum
    by at most 2^-23 = 1.2e-7 relative and a sum of squares by twice that
    (every voxel one ulp off in the same direction); another seed, preset or
    generator moves them far more.  A sum does not see a small edit of a
    single voxel."""
    if not a or not b or set(a) != set(b):
        return False
    for k in a:
        for x, y in zip(a[k], b[k]):
            if abs(x - y) > rel * max(abs(x), abs(y), 1e-300):
                return False
    return True
