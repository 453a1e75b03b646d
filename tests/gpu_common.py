"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import binning

IMG_TOL = 1e-4      # absolute, per channel / depth / alpha (FP32 path vs FP64 oracle)
GRAD_REL = 1e-3     # per-tensor relative L2 error of gradients


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


def compare_images(out, ref, tol=IMG_TOL, pixels=None):
    """Max abs difference of rgb/depth/alpha, excluding pixels whose oracle
    transmittance came within 1e-3 relative of the stop threshold."""
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
    assert err["rgb"] <= tol and err["depth"] <= tol and err["alpha"] <= tol, err
    return err, int((~keep).sum())


def compare_grads(g, ref, rel=GRAD_REL, name=""):
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    e = np.linalg.norm(g - ref) / max(nr, 1e-30)
    assert nr > 0, name
    assert e <= rel, (name, e)
    # elementwise: relative to the element, floored at 1e-3 of the largest
    tol = rel * (np.abs(ref) + 1e-3 * np.abs(ref).max())
    bad = np.abs(g - ref) > 10 * tol
    assert not bad.any(), (name, int(bad.sum()), float(np.abs(g - ref).max()))
    return e
