"""Pins for every slot of the rate controller's statistics words and of its
80 features (oracle/features.py), each from a computation that does not go
through ``block_stats``:

* band energies (words 0..63, features 0..63) are bracketed block by block
  from the exact DCT of Eq. 6 (scipy-pinned) and a rigorous bound on the
  Cordic coefficient error of that very block (the linear-model part scaled
  by the block's own samples, plus the floor-shift truncation part); designed
  cosine-basis blocks at (u0, v0) != (v0, u0) make the brackets tight enough
  that a u/v swap, a wrong shift or a wrong divisor falls outside;
* pixel and gradient statistics (words and features 64..71) come from plain
  loops over the edge-replicated samples (Sec. 2.5.2 works on whole 8x8
  blocks; padding by edge replication);
* the low-AC block fractions (72..75) are counted by brute force over blocks
  designed to sit well inside one energy decade each;
* sizes, target and bias (76..79) from their closed forms.
"""
import math

import numpy as np
import pytest

from oracle import cordic_loeffler, exact_dct, features, linear, spec

SHIFT = spec.P + 1                      # band term (|Y| >> (P + 1))^2
THRESHOLDS = [1 << 10, 1 << 14, 1 << 18, 1 << 22]


def padded_sample(img, y, x):
    """Edge replication: the nearest real sample."""
    h, w = img.shape
    return int(img[min(y, h - 1), min(x, w - 1)])


def padded_blocks(img):
    """List of 8x8 int blocks of the edge-padded plane, block-row major."""
    h, w = img.shape
    nby, nbx = (h + 7) // 8, (w + 7) // 8
    out = []
    for by in range(nby):
        for bx in range(nbx):
            out.append(np.array([[padded_sample(img, by * 8 + i, bx * 8 + j) for j in range(8)] for i in range(8)],
                                dtype=np.int64))
    return out


class Bracket:
    """Per-block bounds on |Y_uv| of the fixed-point forward transform.

    Y_uv = S_uv * Xc_uv with S_uv = 8 * 2^P * g_u * g_v, and
    |Xc_uv - X_uv| <= sum_ij |Cn_ui Cn_vj - C_ui C_vj| |x_ij| + T_uv / S_uv,
    X the exact orthonormal DCT of x = p - 128, Cn the normalised matrix of the
    untruncated graph, T the floor-shift truncation bound in units of Y."""

    def __init__(self):
        g = np.array(cordic_loeffler.gains())
        self.S = 8.0 * (1 << spec.P) * np.outer(g, g)
        cn = linear.normalised_forward()
        c = exact_dct.dct_matrix(8)
        self.M = np.abs(np.kron(cn, cn) - np.kron(c, c))          # (uv, ij)
        self.T = linear.forward_truncation_bound() / self.S

    def abs_y(self, block):
        x = np.asarray(block, dtype=np.float64) - 128.0
        X = exact_dct.dct2(x)
        B = (self.M @ np.abs(x).reshape(64)).reshape(8, 8) + self.T
        # |Y| is an integer: widen by a few float64 ulps, then round inwards
        lo = np.ceil(self.S * np.maximum(np.abs(X) - B, 0.0) * (1.0 - 1e-12) - 1e-9)
        hi = np.floor(self.S * (np.abs(X) + B) * (1.0 + 1e-12) + 1e-9)
        return lo, hi

    def band_terms(self, block):
        """(lo, hi) integer bounds of (|Y_uv| >> (P+1))^2, 8x8 each."""
        lo, hi = self.abs_y(block)
        t_lo = np.floor(lo / (1 << SHIFT)).astype(np.int64)
        t_hi = np.floor(hi / (1 << SHIFT)).astype(np.int64)
        return t_lo * t_lo, t_hi * t_hi


BR = Bracket()


def basis_block(u0, v0, amp, sign=1):
    """128 + amp * (2-D orthonormal cosine basis at (u0, v0)), rounded."""
    c = exact_dct.dct_matrix(8)
    b = 128.0 + sign * amp * np.outer(c[u0], c[v0])
    return np.clip(np.floor(b + 0.5), 0, 255).astype(np.int64)


def assemble(blocks, nbx):
    nby = (len(blocks) + nbx - 1) // nbx
    img = np.full((nby * 8, nbx * 8), 128, dtype=np.uint8)
    for k, b in enumerate(blocks):
        by, bx = divmod(k, nbx)
        img[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8] = b
    return img


def band_bounds(blocks):
    lo = np.zeros((8, 8), dtype=np.int64)
    hi = np.zeros((8, 8), dtype=np.int64)
    for b in blocks:
        a, z = BR.band_terms(b)
        lo += a
        hi += z
    return lo, hi


def test_bracket_holds_on_the_fixed_point_transform():
    """The bracket is a bound on the oracle's own forward output (not a
    definition of it): check it on random and designed blocks."""
    from oracle.codec import forward_coefficients
    rng = np.random.default_rng(3)
    blocks = [rng.integers(0, 256, size=(8, 8)) for _ in range(40)] + \
             [basis_block(u, v, 480, s) for u in range(8) for v in range(8) for s in (1, -1) if u or v]
    for b in blocks:
        y = np.abs(forward_coefficients(np.asarray(b, dtype=np.uint8)[None]))[0]
        lo, hi = BR.abs_y(b)
        assert np.all(y >= lo) and np.all(y <= hi)


# designed plane: strong basis blocks at non-symmetric (u0, v0)
# (no designed pair is the transpose of another designed pair)
DESIGN = [(1, 5, 470, 1), (2, 7, 400, -1), (0, 3, 300, 1), (6, 1, 450, 1), (3, 1, 350, -1), (4, 6, 420, 1),
          (7, 3, 380, -1), (5, 4, 440, 1)]


def designed_plane():
    return assemble([basis_block(u, v, a, s) for u, v, a, s in DESIGN], 4)


@pytest.mark.parametrize("which", ["designed", "ragged_random"])
def test_band_energy_words_and_features_bracketed_by_exact_dct(which):
    if which == "designed":
        img = designed_plane()
    else:
        img = np.random.default_rng(11).integers(0, 256, size=(37, 53)).astype(np.uint8)
    blocks = padded_blocks(img)
    lo, hi = band_bounds(blocks)
    st = features.plane_stats(img)
    f = features.features_from_stats(st, img.shape[1], img.shape[0], 33.0)
    nb = len(blocks)
    for u in range(8):
        for v in range(8):
            w = st[u * 8 + v]
            assert lo[u, v] <= w <= hi[u, v], (u, v, lo[u, v], w, hi[u, v])
            flo, fhi = math.log1p(lo[u, v] / nb), math.log1p(hi[u, v] / nb)
            assert flo - 1e-12 <= f[u * 8 + v] <= fhi + 1e-12, (u, v)


def test_band_energy_brackets_are_tight_enough_to_pin():
    """On the designed plane every designed word's bracket is narrower than a
    factor 4 (a shift by P instead of P + 1) and far above the bracket of its
    transposed word (a u/v swap), and log1p(E / blocks) differs from
    log1p(E / samples) by more than the bracket's width."""
    blocks = padded_blocks(designed_plane())
    lo, hi = band_bounds(blocks)
    nb = len(blocks)
    assert not {(v, u) for u, v, _, _ in DESIGN} & {(u, v) for u, v, _, _ in DESIGN}
    for u, v, _, _ in DESIGN:
        assert hi[u, v] < 4 * lo[u, v], (u, v)
        assert hi[v, u] * 4 < lo[u, v], (u, v)
        assert math.log1p(lo[u, v] / nb) - math.log1p(hi[u, v] / (nb * 64)) > 1.0


def test_low_ac_fraction_words_and_features():
    """Blocks whose AC energy sum_{(u,v) != (0,0)} (|Y_uv| >> (P+1))^2 lies
    well inside one decade: constant blocks (AC exactly 0: every difference
    in the graph is 0), cosine-basis blocks of chosen amplitude, noise."""
    rng = np.random.default_rng(5)
    cats = {0: [np.full((8, 8), c, dtype=np.int64) for c in (0, 77, 128, 255)],
            1: [basis_block(1, 2, 15, 1), basis_block(5, 0, 18, -1)],
            2: [basis_block(3, 6, 60, 1), basis_block(0, 2, 55, -1), basis_block(7, 4, 66, 1)],
            3: [basis_block(2, 5, 250, 1)],
            4: [np.where((np.add.outer(np.arange(8), np.arange(8)) & 1) == 1, 255, 0),      # checkerboard
                np.where(np.arange(8)[None, :] < 4, 20, 235).repeat(8, 0),               # one vertical edge
                rng.integers(0, 2, size=(8, 8)) * 255,                                   # binary noise
                basis_block(1, 7, 480, 1)]}
    blocks, cat_of = [], []
    for c, bs in cats.items():
        for b in bs:
            blocks.append(b)
            cat_of.append(c)
    order = rng.permutation(len(blocks))
    blocks = [blocks[i] for i in order]
    cat_of = [cat_of[i] for i in order]
    # each block's AC energy must be decided by its bracket (design check)
    for b, c in zip(blocks, cat_of):
        lo, hi = BR.band_terms(b)
        if c == 0:
            assert np.all(b == b[0, 0])
            continue
        ac_lo, ac_hi = int(lo.sum() - lo[0, 0]), int(hi.sum() - hi[0, 0])
        bounds = [0] + THRESHOLDS + [1 << 62]
        assert bounds[c] <= ac_lo and ac_hi < bounds[c + 1], (c, ac_lo, ac_hi)
    img = assemble(blocks, 5)
    nb = (img.shape[0] // 8) * (img.shape[1] // 8)
    # assemble() fills any missing blocks with the constant 128
    cat_of = cat_of + [0] * (nb - len(cat_of))
    st = features.plane_stats(img)
    f = features.features_from_stats(st, img.shape[1], img.shape[0], 35.0)
    for k in range(4):
        below = sum(1 for c in cat_of if c <= k)          # energy < 2^(10 + 4k)
        assert st[72 + k] == below, (k, st[72 + k], below)
        assert f[72 + k] == below / nb


@pytest.mark.parametrize("shape,seed", [((37, 53), 1), ((8, 8), 2), ((64, 24), 3), ((5, 130), 4)])
def test_pixel_and_gradient_slots_from_padded_samples(shape, seed):
    h, w = shape
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=shape).astype(np.uint8)
    if seed == 3:
        img[:, :12] = 200                                   # structure: a flat band
    nby, nbx = (h + 7) // 8, (w + 7) // 8
    H, W = nby * 8, nbx * 8
    vals = [padded_sample(img, y, x) for y in range(H) for x in range(W)]
    n = len(vals)
    dxs, dys = [], []
    for by in range(nby):
        for bx in range(nbx):
            for i in range(8):
                for j in range(8):
                    y, x = by * 8 + i, bx * 8 + j
                    if j < 7:
                        dxs.append(padded_sample(img, y, x + 1) - padded_sample(img, y, x))
                    if i < 7:
                        dys.append(padded_sample(img, y + 1, x) - padded_sample(img, y, x))
    st = features.plane_stats(img)
    # integer words
    assert st[64] == sum(vals) and st[65] == sum(v * v for v in vals)
    assert st[66] == min(vals) and st[67] == max(vals)
    assert st[68] == sum(abs(d) for d in dxs) and st[69] == sum(abs(d) for d in dys)
    assert st[70] == sum(d * d for d in dxs) and st[71] == sum(d * d for d in dys)
    assert st[76] == nby * nbx and st[77] == n
    # features: mean and population std over the padded samples (two-pass),
    # mean absolute and RMS within-block differences, sizes, target, bias
    target = 28.0 + seed * 3.3
    f = features.features_from_stats(st, w, h, target)
    mean = sum(vals) / n
    std = math.sqrt(sum((v - mean) ** 2 for v in vals) / n)
    exp = {64: mean / 128.0, 65: std / 64.0, 66: min(vals) / 255.0, 67: max(vals) / 255.0,
           68: sum(abs(d) for d in dxs) / len(dxs) / 32.0, 69: sum(abs(d) for d in dys) / len(dys) / 32.0,
           70: math.sqrt(sum(d * d for d in dxs) / len(dxs)) / 32.0,
           71: math.sqrt(sum(d * d for d in dys) / len(dys)) / 32.0,
           76: math.log(w, 2) / 11.0, 77: math.log(h, 2) / 11.0, 78: (target - 35.0) / 7.0, 79: 1.0}
    for k, v in exp.items():
        assert abs(f[k] - v) <= 1e-12 * max(1.0, abs(v)), (k, f[k], v)
    assert len(dxs) == len(dys) == 56 * nby * nbx


def test_size_slots_distinguish_width_and_height():
    img = np.zeros((16, 1024), dtype=np.uint8)
    f = features.features_from_stats(features.plane_stats(img), 1024, 16, 35.0)
    assert f[76] == 10.0 / 11.0 and f[77] == 4.0 / 11.0 and f[78] == 0.0
