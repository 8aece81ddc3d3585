"""Seeded synthetic grayscale videos shaped like the paper's workloads.

This module only makes inputs; it holds none of the cDMD arithmetic, so both
the FP64 oracle and the CUDA path may draw their inputs from it.

The paper evaluates on surveillance clips (CDnet, BMC; Section 4) that are
not available here.  These clips stand in for them: a static textured
background that is low rank, moving foreground objects, an optional global
illumination drift and per-pixel sensor noise, cut into batches of n frames
(the paper uses 200-frame batches, Section 4.1 "Evaluation settings").

Recipe (all draws from numpy's PCG64 seeded with `seed`):
* background  128 + sum of `n_sinusoids` plane waves
  A sin(2 pi (x cos th + y sin th) / P + ph), A ~ U[5, 25],
  period P ~ U[8, W/2] px, th ~ U[0, pi), ph ~ U[0, 2 pi);
* objects     `n_objects` rectangles (or ellipses), each side ~ U[W/20, W/6],
  constant intensity ~ U[0, 255] redrawn while within 40 of 128,
  speed ~ U[0.5, 3] px/frame in a uniform direction, reflected at the borders;
  a pixel belongs to an object when its centre lies inside it;
* drift       the whole scene is multiplied by 1 + drift * (2 t/(n-1) - 1);
* noise       i.i.d. N(0, noise_sigma^2) per pixel and frame;
* quantise    v = floor(value + 1/2), clamped to [0, 255].

Returns frames in frame-major layout: D[t, j] with pixel j = y W + x, i.e.
the transpose of the paper's m x n video matrix.
"""
import numpy as np

__all__ = ["make_clip", "clip_spec", "truth_from_spec", "Clip", "CONFIGS"]


class Clip:
    """A generated clip: frames (n, m) uint8 and ground truth (n, m) bool."""

    def __init__(self, frames, truth, width, height, seed, params):
        self.frames = frames
        self.truth = truth
        self.width = width
        self.height = height
        self.seed = seed
        self.params = params

    @property
    def m(self):
        return self.width * self.height

    @property
    def n(self):
        return self.frames.shape[0]

    def video_matrix(self):
        """The paper's m x n video matrix (a float64 copy, for the oracle)."""
        return self.frames.T.astype(np.float64)


def _wave_params(rng, W, n_sinusoids):
    """(amplitude, period, orientation, phase) of each background plane wave."""
    waves = []
    for _ in range(n_sinusoids):
        amp = rng.uniform(5.0, 25.0)
        period = rng.uniform(8.0, max(8.0, W / 2.0))
        theta = rng.uniform(0.0, np.pi)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        waves.append((amp, period, theta, phase))
    return np.array(waves, dtype=np.float64).reshape(-1, 4)


def _render_background(waves, W, H):
    y, x = np.mgrid[0:H, 0:W].astype(np.float32)
    bg = np.full((H, W), 128.0, dtype=np.float32)
    for amp, period, theta, phase in waves:
        arg = (x * np.cos(theta) + y * np.sin(theta)) * (2.0 * np.pi / period) + phase
        bg += np.float32(amp) * np.sin(arg).astype(np.float32)
    return bg


def _objects(rng, W, H, n_objects):
    objs = []
    for _ in range(n_objects):
        w = rng.uniform(W / 20.0, W / 6.0)
        h = rng.uniform(W / 20.0, W / 6.0)
        h = min(h, H - 2.0)
        w = min(w, W - 2.0)
        while True:
            inten = rng.uniform(0.0, 255.0)
            if abs(inten - 128.0) >= 40.0:
                break
        cx = rng.uniform(w / 2, W - w / 2)
        cy = rng.uniform(h / 2, H - h / 2)
        speed = rng.uniform(0.5, 3.0)
        ang = rng.uniform(0.0, 2.0 * np.pi)
        objs.append([cx, cy, w, h, inten, speed * np.cos(ang), speed * np.sin(ang)])
    return objs


def _step(obj, W, H):
    cx, cy, w, h, inten, vx, vy = obj
    cx += vx
    cy += vy
    if cx - w / 2 < 0:
        cx, vx = w - cx, -vx
    if cx + w / 2 > W:
        cx, vx = 2 * W - w - cx, -vx
    if cy - h / 2 < 0:
        cy, vy = h - cy, -vy
    if cy + h / 2 > H:
        cy, vy = 2 * H - h - cy, -vy
    obj[:] = [cx, cy, w, h, inten, vx, vy]


def _cover(obj, W, H, shape):
    """Boolean coverage (pixel centres inside the object) and its bbox."""
    cx, cy, w, h = obj[:4]
    x0 = max(int(np.floor(cx - w / 2)), 0)
    x1 = min(int(np.ceil(cx + w / 2)) + 1, W)
    y0 = max(int(np.floor(cy - h / 2)), 0)
    y1 = min(int(np.ceil(cy + h / 2)) + 1, H)
    ys = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5
    xs = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5
    if shape == "ellipse":
        inside = ((xs - cx) / (w / 2)) ** 2 + ((ys - cy) / (h / 2)) ** 2 <= 1.0
    else:
        inside = (np.abs(xs - cx) <= w / 2) & (np.abs(ys - cy) <= h / 2)
    return inside, (y0, y1, x0, x1)


def _trajectories(objs, n, W, H):
    """Object states (cx, cy, w, h, intensity) at frames 0..n-1 (n x objects x 5)."""
    objs = [list(o) for o in objs]
    out = np.zeros((n, len(objs), 5))
    for t in range(n):
        for q, obj in enumerate(objs):
            out[t, q] = obj[:5]
            _step(obj, W, H)
    return out


def clip_spec(width, height, n, seed, n_sinusoids=6, n_objects=3, shape="rectangle", drift=0.0,
              noise_sigma=3.0):
    """The scene parameters make_clip draws for `seed`: plane waves
    (n_sinusoids x [amplitude, period, orientation, phase]) and object states
    per frame (n x n_objects x [cx, cy, w, h, intensity]).  A renderer that
    draws its own noise can rebuild the clip's scene from them."""
    rng = np.random.default_rng(seed)
    W, H = int(width), int(height)
    waves = _wave_params(rng, W, n_sinusoids)
    objs = _objects(rng, W, H, n_objects)
    return dict(width=W, height=H, n=int(n), waves=waves, objects=_trajectories(objs, n, W, H), shape=shape,
                drift=float(drift), noise_sigma=float(noise_sigma))


def make_clip(width, height, n, seed, n_sinusoids=6, n_objects=3,
              shape="rectangle", drift=0.0, noise_sigma=3.0):
    """Generate one clip; see the module docstring for the recipe."""
    rng = np.random.default_rng(seed)
    W, H = int(width), int(height)
    waves = _wave_params(rng, W, n_sinusoids)
    bg = _render_background(waves, W, H)
    objs = _objects(rng, W, H, n_objects)
    states = _trajectories(objs, n, W, H)
    frames = np.empty((n, H * W), dtype=np.uint8)
    truth = np.zeros((n, H * W), dtype=bool)
    for t in range(n):
        scene = bg.copy()
        tmask = np.zeros((H, W), dtype=bool)
        for state in states[t]:
            inside, (y0, y1, x0, x1) = _cover(state, W, H, shape)
            scene[y0:y1, x0:x1][inside] = state[4]
            tmask[y0:y1, x0:x1] |= inside
        if drift != 0.0 and n > 1:
            scene *= np.float32(1.0 + drift * (2.0 * t / (n - 1) - 1.0))
        if noise_sigma > 0.0:
            scene += rng.standard_normal((H, W), dtype=np.float32) * np.float32(noise_sigma)
        frames[t] = np.clip(np.floor(scene + 0.5), 0, 255).astype(np.uint8).reshape(-1)
        truth[t] = tmask.reshape(-1)
    params = dict(n_sinusoids=n_sinusoids, n_objects=n_objects, shape=shape,
                  drift=drift, noise_sigma=noise_sigma)
    return Clip(frames, truth, W, H, seed, params)


def truth_from_spec(spec):
    """Ground-truth foreground (n, m) bool of the clip a spec describes: the
    pixels whose centre lies inside an object in that frame (what make_clip
    returns as truth), without rendering the frames."""
    W, H, n = spec["width"], spec["height"], spec["n"]
    truth = np.zeros((n, H * W), dtype=bool)
    for t in range(n):
        tmask = np.zeros((H, W), dtype=bool)
        for state in spec["objects"][t]:
            inside, (y0, y1, x0, x1) = _cover(state, W, H, spec["shape"])
            tmask[y0:y1, x0:x1] |= inside
        truth[t] = tmask.reshape(-1)
    return truth


# Workload shapes (width, height, n, generator options, method parameters).
CONFIGS = {
    "plain_160x120x100": dict(width=160, height=120, n=100, gen=dict(),
                              k=200, r=10, K=10, tau=25.0, ctype="gaussian"),
    "precision_1080p_x200": dict(width=1920, height=1080, n=200, gen=dict(drift=0.1),
                                 k=1000, r=20, K=10, tau=25.0, ctype="gaussian"),
    "gather_4k_x300": dict(width=3840, height=2160, n=300,
                           gen=dict(n_objects=8, shape="ellipse"),
                           k=1000, r=30, K=10, tau=25.0, ctype="sparse",
                           density=1e-3),
}
