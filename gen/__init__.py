"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random numbers and arranges them into columns and
images.  It holds none of the method's arithmetic: no predicate, join,
aggregate, soft operator or network layer is evaluated here.  Every draw uses
``numpy.random.Generator(PCG64)`` keyed by ``SeedSequence([seed, stream])`` so
that any column can be regenerated on its own.

Workload shapes (all synthetic; the paper's own datasets are not available):

* fact table: decision-support "line item" shape -- int32 key, int8 flag
  (0..2), int8 status (0..1), int64 quantity in hundredths U[100,5000], int64
  price in cents U[90000,10500000], int64 discount in hundredths U[0,10],
  int32 date in days U[0,2556].
* dimension table: unique shuffled int32 keys 1..n, int8 segment U[0,4],
  int32 date U[0,2556].
* three-table join chain: probe rows with Zipf(1.0) foreign keys over the
  build table, build rows with Zipf(0.5) foreign keys over a third table,
  int64 payloads U[0,1e9], int32 categories U[0,99999].
* soft-query rows: fp32 x ~ N(0,1), fp32 v ~ U[0,100], int32 group id.
* string columns (offsets + bytes): rows drawn from a seeded vocabulary of
  random lower-case words, some of them prefixes of others.
* N:M join tables: build keys with a fixed number of rows per distinct key
  on average (Poisson), probe keys uniform over a wider range.
* LLP rows (stand-in for the paper's Adult Income census rows, Sec. 5.3):
  six standardised fp32 numeric features shaped like the census numeric
  columns (an age-like and an hours-like Gaussian, a discrete education
  level, two mostly-zero heavy-tailed capital columns, an uninformative
  sampling weight) and an int32 binary label, about 24% positive, from a
  fixed logistic model of the features.  Rows are in random order, so bags
  of consecutive rows are random bags.  Standard Laplace draws for the
  label-DP counts come from a stream of their own.
* ranked groups (soft ORDER BY ... LIMIT k): fp32 scores x ~ N(0,1), fp32
  payloads v ~ U[0,100], groups of consecutive rows whose sizes are uniform
  on [size/2, 3 size/2] (int64 offsets).
* glyph grids: 4x4 cells of 28x28 uint8 glyphs drawn from 10 seeded stroke
  templates with affine jitter and Gaussian noise (stand-in for the paper's
  MNIST grids, Sec. 5.5).
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

BASE_SEED = 20221106

FACT_COLS = ("key", "flag", "status", "qty", "price", "disc", "date")
DIM_COLS = ("key", "segment", "date")


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def _uniform_int(seed, stream, lo, hi, n, dtype):
    """Integers uniform on the closed range [lo, hi]."""
    return rng(seed, stream).integers(lo, hi + 1, size=n, dtype=np.int64).astype(dtype, copy=False)


def fact_table(n: int, key_max: int, seed: int, cols=FACT_COLS) -> dict:
    """Fact table columns (structure of arrays, one numpy array per column)."""
    spec = {
        "key": (1, 1, key_max, np.int32),
        "flag": (2, 0, 2, np.int8),
        "status": (3, 0, 1, np.int8),
        "qty": (4, 100, 5000, np.int64),
        "price": (5, 90000, 10500000, np.int64),
        "disc": (6, 0, 10, np.int64),
        "date": (7, 0, 2556, np.int32),
    }
    out = {}
    for c in cols:
        stream, lo, hi, dt = spec[c]
        out[c] = _uniform_int(seed, stream, lo, hi, n, dt)
    return out


def permutation_keys(n: int, seed: int, stream: int) -> np.ndarray:
    """The keys 1..n in a seeded random order (int32)."""
    p = rng(seed, stream).permutation(n).astype(np.int32)
    p += 1
    return p


def dim_table(n: int, seed: int, cols=DIM_COLS) -> dict:
    out = {}
    if "key" in cols:
        out["key"] = permutation_keys(n, seed, 11)
    if "segment" in cols:
        out["segment"] = _uniform_int(seed, 12, 0, 4, n, np.int8)
    if "date" in cols:
        out["date"] = _uniform_int(seed, 13, 0, 2556, n, np.int32)
    return out


def zipf_ranks(n_samples: int, domain: int, s: float, seed: int, stream: int) -> np.ndarray:
    """Bounded Zipf ranks in 1..domain with P(r) proportional to r**-s.

    Inverse-CDF sampling: uniforms from PCG64 located in the float64
    cumulative table with searchsorted (chunked over threads; numpy releases
    the GIL there).
    """
    w = np.arange(1, domain + 1, dtype=np.float64) ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng(seed, stream).random(n_samples)
    chunks = np.array_split(u, max(1, min(64, n_samples // 1_000_000 + 1)))
    with ThreadPoolExecutor(8) as ex:
        parts = list(ex.map(lambda c: np.searchsorted(cdf, c, side="right"), chunks))
    r = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    np.minimum(r, domain - 1, out=r)
    return (r + 1).astype(np.int64)


def chain_tables(n_probe: int, n_build: int, n_third: int, seed: int,
                 s_probe: float = 1.0, s_build: float = 0.5, n_category: int = 100000) -> dict:
    """Three-table join chain: probe.fk -> build.pk, build.fk2 -> third.pk.

    Zipf ranks are mapped to keys through a seeded permutation so that hot keys
    are scattered over the key range.
    """
    third_pk = permutation_keys(n_third, seed, 21)
    third_cat = _uniform_int(seed, 22, 0, n_category - 1, n_third, np.int32)
    build_pk = permutation_keys(n_build, seed, 23)
    rank_to_third = permutation_keys(n_third, seed, 24)
    build_fk2 = rank_to_third[zipf_ranks(n_build, n_third, s_build, seed, 25) - 1]
    rank_to_build = permutation_keys(n_build, seed, 26)
    probe_fk = rank_to_build[zipf_ranks(n_probe, n_build, s_probe, seed, 27) - 1]
    payload = _uniform_int(seed, 28, 0, 1_000_000_000, n_probe, np.int64)
    return {
        "third_pk": third_pk, "third_cat": third_cat,
        "build_pk": build_pk, "build_fk2": build_fk2,
        "probe_fk": probe_fk, "probe_payload": payload,
    }


def soft_table(n: int, n_groups: int, seed: int) -> dict:
    """Rows for the differentiable soft filter / soft aggregation query."""
    x = rng(seed, 31).standard_normal(n, dtype=np.float32)
    v = (rng(seed, 32).random(n, dtype=np.float32) * np.float32(100.0)).astype(np.float32)
    gid = _uniform_int(seed, 33, 0, n_groups - 1, n, np.int32)
    return {"x": x, "v": v, "gid": gid}


# ---------------------------------------------------------------------------
# glyph grids (stand-in for MNISTGrid)
# ---------------------------------------------------------------------------

CELL = 28
GRID = 4
N_CLASSES = 10


def stroke_templates(seed: int = BASE_SEED + 4) -> list:
    """10 seeded polylines of 2..4 strokes inside a 20x20 box (pixel units,
    origin at the box centre).  Returned as a list of (P, 2) float64 arrays of
    polyline vertices (P = strokes + 1)."""
    g = rng(seed, 41)
    out = []
    for _k in range(N_CLASSES):
        n_strokes = int(g.integers(2, 5))
        pts = g.uniform(-10.0, 10.0, size=(n_strokes + 1, 2))
        out.append(pts)
    return out


def _render(points: np.ndarray, valid: np.ndarray) -> np.ndarray:
    """Anti-aliased polylines of width 2 px.

    points: (B, P, 2) vertices in cell pixel coordinates; valid: (B, P-1) bool
    mask of real segments.  Returns float intensities (B, 28, 28) in [0, 1].
    """
    ys, xs = np.meshgrid(np.arange(CELL) + 0.5, np.arange(CELL) + 0.5, indexing="ij")
    pix = np.stack([xs.ravel(), ys.ravel()], axis=1)  # (784, 2) as (x, y)
    a = points[:, :-1, None, :]  # (B, S, 1, 2)
    b = points[:, 1:, None, :]
    ab = b - a
    ap = pix[None, None, :, :] - a  # (B, S, 784, 2)
    denom = np.maximum((ab * ab).sum(-1), 1e-12)
    t = np.clip((ap * ab).sum(-1) / denom, 0.0, 1.0)
    d = np.sqrt(((ap - t[..., None] * ab) ** 2).sum(-1))  # (B, S, 784)
    d = np.where(valid[:, :, None], d, np.inf)
    dmin = d.min(axis=1)
    inten = np.clip(1.0 - (dmin - 1.0), 0.0, 1.0)  # half width 1 px, 1 px ramp
    return inten.reshape(-1, CELL, CELL)


def glyph_cells(labels: np.ndarray, seed: int, stream: int, sizes: np.ndarray | None = None) -> np.ndarray:
    """Render one 28x28 uint8 glyph per label (labels: 1-d int array).  With
    `sizes` (1-d 0/1 array) a size-0 glyph is drawn at scale 0.55..0.70 and a
    size-1 glyph at 0.95..1.15 instead of 0.85..1.15."""
    templates = stroke_templates()
    n = labels.shape[0]
    g = rng(seed, stream)
    rot = np.deg2rad(g.uniform(-15.0, 15.0, n))
    scale = g.uniform(0.85, 1.15, n)
    if sizes is not None:
        u = (scale - 0.85) / 0.30  # the same draw, mapped into the size's range
        scale = np.where(np.asarray(sizes) == 0, 0.55 + 0.15 * u, 0.95 + 0.20 * u)
    shear = g.uniform(-0.15, 0.15, n)
    shift = g.uniform(-2.0, 2.0, (n, 2))
    noise_g = rng(seed, stream + 1)
    pmax = max(t.shape[0] for t in templates)
    pts = np.zeros((n, pmax, 2))
    valid = np.zeros((n, pmax - 1), dtype=bool)
    for k, t in enumerate(templates):
        sel = labels == k
        pts[sel, : t.shape[0]] = t
        pts[sel, t.shape[0]:] = t[-1]
        valid[sel, : t.shape[0] - 1] = True
    c, s_ = np.cos(rot), np.sin(rot)
    # A = R(rot) @ Shear(shear) @ diag(scale)
    a00 = c * scale
    a01 = (c * shear - s_) * scale
    a10 = s_ * scale
    a11 = (s_ * shear + c) * scale
    x, y = pts[..., 0], pts[..., 1]
    tx = a00[:, None] * x + a01[:, None] * y + CELL / 2 + shift[:, 0:1]
    ty = a10[:, None] * x + a11[:, None] * y + CELL / 2 + shift[:, 1:2]
    pts = np.stack([tx, ty], axis=-1)
    out = np.empty((n, CELL, CELL), dtype=np.uint8)
    step = 2048
    for i in range(0, n, step):
        inten = _render(pts[i:i + step], valid[i:i + step])
        inten = inten + noise_g.normal(0.0, 0.1, inten.shape)
        out[i:i + step] = np.rint(np.clip(inten, 0.0, 1.0) * 255.0).astype(np.uint8)
    return out


def glyph_grids(n_grids: int, seed: int, stream: int = 50) -> tuple:
    """``n_grids`` grid images of 4x4 glyph cells.

    Returns (images uint8 [n_grids, 112, 112], labels int64 [n_grids, 4, 4]).
    The image layout is the grid as a picture; cell (r, c) of grid n is
    ``images[n, 28r:28r+28, 28c:28c+28]``.
    """
    labels = rng(seed, stream).integers(0, N_CLASSES, size=(n_grids, GRID, GRID), dtype=np.int64)
    cells = glyph_cells(labels.reshape(-1), seed, stream + 1)
    img = cells.reshape(n_grids, GRID, GRID, CELL, CELL).transpose(0, 1, 3, 2, 4)
    img = np.ascontiguousarray(img).reshape(n_grids, GRID * CELL, GRID * CELL)
    return img, labels


def glyph_grids_sized(n_grids: int, seed: int, stream: int = 80) -> tuple:
    """Grid images like glyph_grids whose cells also carry a size attribute
    (0 small, 1 large; the second attribute of the paper's Digit x Size
    grouping).  Returns (images uint8 [n, 112, 112], digits int64 [n, 4, 4],
    sizes int64 [n, 4, 4])."""
    labels = rng(seed, stream).integers(0, N_CLASSES, size=(n_grids, GRID, GRID), dtype=np.int64)
    sizes = rng(seed, stream + 2).integers(0, 2, size=(n_grids, GRID, GRID), dtype=np.int64)
    cells = glyph_cells(labels.reshape(-1), seed, stream + 1, sizes=sizes.reshape(-1))
    img = cells.reshape(n_grids, GRID, GRID, CELL, CELL).transpose(0, 1, 3, 2, 4)
    img = np.ascontiguousarray(img).reshape(n_grids, GRID * CELL, GRID * CELL)
    return img, labels, sizes


def size_head_params(seed: int) -> dict:
    """Initial weights of the 2-class size head on the CNN's 128 hidden
    units: fc2s w [2, 128], b [2], Kaiming-uniform like cnn_params."""
    g = rng(seed, 90)
    bound = math.sqrt(6.0 / 128)
    bb = 1.0 / math.sqrt(128)
    return {"fc2s_w": g.uniform(-bound, bound, (2, 128)).astype(np.float32),
            "fc2s_b": rng(seed, 91).uniform(-bb, bb, 2).astype(np.float32)}


def cnn_params(seed: int) -> dict:
    """Kaiming-uniform initial weights for the 4-layer glyph CNN, as fp32.

    Layouts: conv1 w [32, 3, 3] (one input channel), conv2 w [64, 3, 3, 32]
    (out, ky, kx, in), fc1 w [128, 9216] with inputs flattened in (y, x, c)
    order of the pooled 12x12x64 map, fc2 w [10, 128].  Biases start at
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)).
    """
    shapes = {
        "conv1_w": ((32, 3, 3), 9), "conv1_b": ((32,), 9),
        "conv2_w": ((64, 3, 3, 32), 288), "conv2_b": ((64,), 288),
        "fc1_w": ((128, 9216), 9216), "fc1_b": ((128,), 9216),
        "fc2_w": ((10, 128), 128), "fc2_b": ((10,), 128),
    }
    out = {}
    for i, (name, (shape, fan_in)) in enumerate(shapes.items()):
        g = rng(seed, 60 + i)
        if name.endswith("_w"):
            bound = math.sqrt(6.0 / fan_in)  # Kaiming-uniform, ReLU gain
        else:
            bound = 1.0 / math.sqrt(fan_in)
        out[name] = g.uniform(-bound, bound, size=shape).astype(np.float32)
    return out


# ---------------------------------------------------------------------------
# string columns and N:M join tables
# ---------------------------------------------------------------------------

def vocabulary(n_words: int, seed: int, min_len: int = 1, max_len: int = 24) -> list:
    """n_words distinct random lower-case byte strings; about one in ten is a
    proper prefix of another word of the list."""
    r = rng(seed, 61)
    words = set()
    out = []
    while len(out) < n_words:
        ln = int(r.integers(min_len, max_len + 1))
        w = bytes(r.integers(97, 123, ln, dtype=np.int64).astype(np.uint8))
        if out and r.random() < 0.1:
            base = out[int(r.integers(0, len(out)))]
            if len(base) > 1:
                w = base[:int(r.integers(1, len(base)))]
        if w not in words:
            words.add(w)
            out.append(w)
    return out


def string_column(n: int, n_words: int, seed: int, max_len: int = 24):
    """An offsets + bytes column of n rows drawn uniformly from a vocabulary
    of n_words words.  Returns (offsets int32[n+1], bytes uint8, vocabulary,
    row word index int64[n])."""
    vocab = vocabulary(n_words, seed, 1, max_len)
    idx = rng(seed, 62).integers(0, n_words, n, dtype=np.int64)
    lens = np.array([len(w) for w in vocab], np.int64)[idx]
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    pool = np.frombuffer(b"".join(vocab), dtype=np.uint8)
    starts = np.zeros(n_words + 1, np.int64)
    np.cumsum([len(w) for w in vocab], out=starts[1:])
    # row bytes: the vocabulary word's bytes, row after row
    src = np.repeat(starts[idx], lens) + (np.arange(offsets[-1]) - np.repeat(offsets[:-1], lens))
    data = pool[src] if len(src) else np.zeros(0, np.uint8)
    return offsets.astype(np.int32), data.astype(np.uint8), vocab, idx


def nm_join_tables(n_build: int, n_probe: int, dup: float, seed: int) -> dict:
    """Build keys in 1..K with K = n_build / dup (about dup rows per key),
    probe keys uniform in 1..2K (half of them match), int64 payloads."""
    k = max(1, int(n_build / dup))
    return {
        "build_key": _uniform_int(seed, 71, 1, k, n_build, np.int32),
        "build_pay": _uniform_int(seed, 72, 0, 1_000_000, n_build, np.int64),
        "probe_key": _uniform_int(seed, 73, 1, 2 * k, n_probe, np.int32),
        "probe_date": _uniform_int(seed, 74, 0, 2556, n_probe, np.int32),
    }


LLP_FEATURES = 6
# the fixed logistic model that draws the labels (weights per standardised
# feature, then the intercept that puts about 24% of rows in class 1)
_LLP_W = np.array([0.9, 0.1, 1.1, 0.8, 0.35, 0.6])
_LLP_B = -1.75


def llp_table(n: int, seed: int, stream: int = 120) -> tuple:
    """Census-shaped rows for learning from label proportions: features fp32
    [n, 6] (each column standardised to mean 0, variance 1 over the drawn
    rows; a column with no spread is only centred), labels int32 [n] in
    {0, 1}."""
    g = rng(seed, stream)
    age = g.normal(38.6, 13.6, n)
    fnl = np.log(g.lognormal(12.0, 0.5, n))  # sampling weight: no relation to the label
    edu = np.clip(np.rint(g.normal(10.1, 2.6, n)), 1, 16)
    gain = np.where(g.random(n) < 0.08, np.log1p(g.lognormal(8.5, 1.0, n)), 0.0)
    loss = np.where(g.random(n) < 0.05, np.log1p(g.lognormal(7.5, 0.3, n)), 0.0)
    hours = np.clip(g.normal(40.4, 12.3, n), 1, 99)
    raw = np.stack([age, fnl, edu, gain, loss, hours], axis=1)
    sd = raw.std(axis=0)
    sd[sd == 0] = 1.0  # a single row (or a constant column) stays finite
    X = (raw - raw.mean(axis=0)) / sd
    z = X @ _LLP_W + _LLP_B + g.logistic(0.0, 1.0, n)
    y = (z > 0).astype(np.int32)
    return X.astype(np.float32), y


def laplace_noise(n_bags: int, k: int, seed: int, stream: int = 130) -> np.ndarray:
    """Standard Laplace draws (location 0, scale 1), fp32 [n_bags, k]: the
    random numbers of the label-DP mechanism, scaled by the method."""
    return rng(seed, stream).laplace(0.0, 1.0, (n_bags, k)).astype(np.float32)


def ranked_groups(n_groups: int, size: int, seed: int, stream: int = 140) -> dict:
    """Groups of consecutive rows for a per-group ORDER BY ... LIMIT k: x fp32
    N(0,1) scores, v fp32 U[0,100] payloads, offsets int64 [n_groups + 1]
    with group sizes uniform on [size // 2, size + size // 2]."""
    g = rng(seed, stream)
    sizes = g.integers(max(1, size // 2), size + size // 2 + 1, n_groups)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    return {"x": g.standard_normal(n).astype(np.float32), "v": g.uniform(0, 100, n).astype(np.float32),
            "offsets": offsets}
