"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import binning

IMG_TOL = 1e-4      # absolute, per channel / depth / alpha (FP32 path vs FP64 oracle)
GRAD_REL = 1e-3     # gradients: per-tensor relative L2 error, and elementwise
                    # |g - g*| <= GRAD_REL (|g*| + 1e-3 max |g*|)
# Pixels whose termination is rounding-sensitive (oracle.NEAR_STOP_REL) are
# left out of image comparisons; at most this fraction of the compared
# pixels (and at least 3 of them) may be left out.
NEAR_STOP_MAX_FRAC = 1e-3


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2412_04459_gb300 import build
    build.build()


def run_gpu(scene, cam, K=1, t_stop=1e-4, bg=(0.0, 0.0, 0.0), capacity=None, inspect=True):
    from paper_2412_04459_gb300 import DeviceScene, Frame
    dev = DeviceScene.from_host(scene)
    fr = Frame(dev, cam, K=K, t_stop=t_stop, bg=bg, pair_capacity=capacity)
    fr.preprocess()
    fr.bin_sort()
    out = fr.forward()
    ins = fr.inspect() if inspect else None
    return fr, out, ins


def to_np(out):
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def compare_integers(scene, cam, ins, tile=16):
    """Bit-exact comparison of tile masks, Morton codes, rectangles, counts,
    sorted keys/values and ranges, outside the oracle's rounding-sensitive
    ("either") cases.  Returns the number of excluded voxels and tiles."""
    masks, t_either = binning.tile_masks(cam, tile)
    assert (ins["tile_mask"][~t_either] == masks[~t_either]).all()
    code, ok = binning.voxel_octpath(scene)
    assert ok.all()
    assert (ins["octpath"] == code).all()
    rect, amb = binning.voxel_rects(scene, cam, tile)
    g_rect = ins["rect"].astype(np.int64)
    same = (g_rect == rect).all(1)
    assert same[~amb].all(), np.where(~same & ~amb)[0][:10]
    assert (np.abs(g_rect - rect)[~same] <= 1).all()
    # pairs: drop voxels whose rectangle differs and tiles whose mask is ambiguous
    keys, vals, counts = binning.emit_pairs(scene, cam, tile, masks=ins["tile_mask"], rects=g_rect)
    sk, sv = binning.sort_pairs(keys, vals)
    assert ins["n_pairs"] == len(sk)
    assert (ins["count"] == counts).all()
    assert (ins["keys"] == sk).all()
    assert (ins["values"] == sv).all()
    ntx, nty = binning.tile_grid(cam, tile)
    assert (ins["ranges"].astype(np.int64) == binning.tile_ranges(sk, ntx * nty)).all()
    # the oracle's own masks/rects give the same pair set where unambiguous
    ok_t = ~t_either
    okv = same
    keys_o, vals_o, _ = binning.emit_pairs(scene, cam, tile, masks=masks, rects=rect)
    sko, svo = binning.sort_pairs(keys_o, vals_o)
    sel_o = okv[(svo & 0x1FFFFFFF).astype(np.int64)] & ok_t[(sko >> np.uint64(48)).astype(np.int64)]
    sel_g = okv[(sv & 0x1FFFFFFF).astype(np.int64)] & ok_t[(sk >> np.uint64(48)).astype(np.int64)]
    assert (sko[sel_o] == sk[sel_g]).all() and (svo[sel_o] == sv[sel_g]).all()
    return int((~same).sum()), int(t_either.sum())


def near_stop_allowance(n):
    return max(3, int(NEAR_STOP_MAX_FRAC * n))


def compare_images(out, ref, tol=IMG_TOL, pixels=None):
    """Max abs difference of rgb/depth/alpha, excluding the pixels whose
    oracle transmittance came within oracle.NEAR_STOP_REL (relative) of the
    stop threshold; their number is asserted small.  Returns (errors,
    number excluded)."""
    o = to_np(out)
    if pixels is None:
        keep = ref["near_stop"] == 0
        rgb = o["rgb"][:, keep]
        rgb_ref = ref["rgb"][:, keep]
        dep, dep_ref = o["depth"][keep], ref["depth"][keep]
        alp, alp_ref = o["alpha"][keep], ref["alpha"][keep]
    else:
        x, y = pixels[:, 0], pixels[:, 1]
        keep = ref["near_stop"] == 0
        rgb = o["rgb"][:, y, x][:, keep]
        rgb_ref = ref["rgb"].T[:, keep]
        dep, dep_ref = o["depth"][y, x][keep], ref["depth"][keep]
        alp, alp_ref = o["alpha"][y, x][keep], ref["alpha"][keep]
    err = dict(rgb=float(np.abs(rgb - rgb_ref).max(initial=0.0)),
               depth=float(np.abs(dep - dep_ref).max(initial=0.0)),
               alpha=float(np.abs(alp - alp_ref).max(initial=0.0)))
    n_out = int((~keep).sum())
    print(f"PARITY image: {err}, near-stop excluded {n_out} of {keep.size}")
    assert err["rgb"] <= tol and err["depth"] <= tol and err["alpha"] <= tol, (err, n_out)
    assert n_out <= near_stop_allowance(keep.size), (n_out, keep.size)
    return err, n_out


# Elementwise, an FP32 gradient element is only as exact as the terms it
# sums.  Two FP32 effects, measured per pixel against the oracle, set how
# exact a term is: (1) ~3e-5 .. 8e-5 relative in every term (the larger where
# the transmittance in front of the voxel is ~1e-69), which matters where an
# element's terms of both signs cancel (sums of |term| up to 1000x the
# element); (2) a grazing hit's segment length l = (b - a)|r_d| is the
# difference of two FP32 ray distances, each from an FP32 plane coordinate
# relative to the camera divided by a direction component, so its terms
# carry a relative error of order 2^-24 times the length's condition number
# kappa (the oracle's segment_condition; measured: 2 % on a 1.6e-5-long
# segment at depth 2.7, 7e-4 on a 6.6e-3-long one crossing planes at a
# shallow angle, both below 2^-24 kappa).  The bound adds COND_REL times the
# oracle's sum of |term| and SEG_REL times its sum of kappa |term|.
COND_REL = 1e-4
SEG_REL = 4 * 2.0 ** -24


def oracle_grads(scene, cam, g_rgb, g_depth, g_alpha, **kw):
    """The oracle's (d_grid, d_sh) and their contribution magnitudes."""
    mag = {}
    og, osh = oracle.render_grad(scene, cam, g_rgb, g_depth, g_alpha, magnitudes=mag, **kw)
    return og, osh, mag


def compare_grads(g, ref, rel=GRAD_REL, name="", mag=None):
    """Per tensor ||g - g*|| <= rel ||g*||; elementwise |g - g*| <= rel (|g*|
    + 1e-3 max |g*|) + COND_REL mag + SEG_REL mag_seg, (mag, mag_seg) the
    oracle's magnitudes of the element's terms (required)."""
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    assert mag is not None, name
    mag, mag_seg = (np.asarray(m, np.float64).reshape(-1) for m in mag)
    nr = np.linalg.norm(ref)
    e = np.linalg.norm(g - ref) / max(nr, 1e-30)
    assert nr > 0, name
    assert e <= rel, (name, e)
    # elementwise: relative to the element, floored at 1e-3 of the largest,
    # plus the rounding the element's cancelling contributions carry
    tol = rel * (np.abs(ref) + 1e-3 * np.abs(ref).max()) + COND_REL * mag + SEG_REL * mag_seg
    ratio = np.abs(g - ref) / tol
    bad = ratio > 1.0
    worst = int(np.argmax(ratio))
    print(f"PARITY grad {name}: rel L2 {e:.3e}, worst elementwise ratio {float(ratio[worst]):.3f}")
    assert not bad.any(), (name, "elementwise", int(bad.sum()), float(ratio[worst]), worst, float(g[worst]),
                           float(ref[worst]))
    return e


# The same FP32 gradient sums accumulated in another order (atomics from
# other warps, views summed per sort partition) differ by rounding only:
# elementwise |a - b| <= REORDER_REL (|b| + 1e-3 max |b|).
REORDER_REL = 1e-4


def compare_reordered(a, b, name=""):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    tol = REORDER_REL * (np.abs(b) + 1e-3 * np.abs(b).max())
    ratio = np.abs(a - b) / tol
    worst = int(np.argmax(ratio))
    print(f"PARITY reordered {name}: worst elementwise ratio {float(ratio[worst]):.3f}")
    assert (ratio <= 1.0).all(), (name, int((ratio > 1).sum()), float(ratio[worst]), float(a[worst]), float(b[worst]))
