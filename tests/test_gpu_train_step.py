"""The training step of the 1M-voxel workload, checked on a 4096-voxel
sub-scene: the MSE loss against a target rendered from perturbed densities,
its gradients with respect to the corner densities and the SH coefficients
through rasterize() (the CUDA forward and backward), against FP64 central
finite differences of the oracle's loss."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import require_gpu

pytestmark = pytest.mark.gpu

N_SUB = 4096


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _sub_scene():
    """The 4096 voxels of the 1M shell scene nearest to the point where the
    shell crosses the -z axis through its centre, and a narrow camera on it."""
    scene = cached("shell1m", lambda: synth.shell_scene(seed=0))
    p = np.array([0.5, 0.5, 0.1])
    near = np.argsort(np.linalg.norm(scene.centre.astype(np.float64) - p, axis=1))[:N_SUB]
    sub = synth.subscene(scene, np.sort(near))
    cam = synth.look_at((0.5, 0.5, -0.6), (0.5, 0.5, 0.1), (0, 1, 0), 6, 96, 96)
    return sub, cam


def test_training_step_gradients_match_finite_differences():
    import torch
    from paper_2412_04459_gb300 import DeviceScene, rasterize
    sub, cam = cached("train_sub", _sub_scene)
    assert sub.n_vox == N_SUB
    K, t_stop = 3, 0.0          # no early termination: the loss is smooth in every parameter
    rng = np.random.default_rng(3)
    grid64 = sub.grid.astype(np.float64)
    sh64 = sub.sh.astype(np.float64)
    target = oracle.render(sub, cam, K=K, t_stop=t_stop,
                           grid=grid64 + 0.1 * rng.normal(size=grid64.shape))["rgb"]
    assert np.ptp(target) > 0.01

    def loss64(grid=grid64, sh=sh64):
        c = oracle.render(sub, cam, K=K, t_stop=t_stop, grid=grid, sh=sh)["rgb"]
        return float(np.mean((c - target) ** 2))

    dev = DeviceScene.from_host(sub)
    grid = dev.grid.clone().requires_grad_(True)
    sh = dev.sh.clone().requires_grad_(True)
    rgb, _, _ = rasterize(grid, sh, dev, cam, K=K, t_stop=t_stop)
    loss = ((rgb - torch.as_tensor(target, dtype=torch.float32, device="cuda")) ** 2).mean()
    loss.backward()
    g_grid = grid.grad.detach().cpu().numpy().astype(np.float64)
    g_sh = sh.grad.detach().cpu().numpy().astype(np.float64).reshape(-1)
    assert abs(float(loss.detach()) - loss64()) <= 1e-5 * loss64() + 1e-9

    # finite differences on the grid points and SH coefficients with the
    # largest gradients plus a few random ones
    h = 1e-4
    pick_g = np.unique(np.concatenate([np.argsort(-np.abs(g_grid))[:16],
                                       rng.choice(np.nonzero(g_grid)[0], 8, replace=False)]))
    pick_s = np.unique(np.concatenate([np.argsort(-np.abs(g_sh))[:16],
                                       rng.choice(np.nonzero(g_sh)[0], 8, replace=False)]))
    fd_g, fd_s = [], []
    for i in pick_g:
        gp, gm = grid64.copy(), grid64.copy()
        gp[i] += h
        gm[i] -= h
        fd_g.append((loss64(grid=gp) - loss64(grid=gm)) / (2 * h))
    for j in pick_s:
        sp, sm = sh64.copy().reshape(-1), sh64.copy().reshape(-1)
        sp[j] += h
        sm[j] -= h
        fd_s.append((loss64(sh=sp.reshape(sh64.shape)) - loss64(sh=sm.reshape(sh64.shape))) / (2 * h))
    for gpu, fd, name in ((g_grid[pick_g], np.array(fd_g), "grid"), (g_sh[pick_s], np.array(fd_s), "sh")):
        rel = np.linalg.norm(gpu - fd) / np.linalg.norm(fd)
        assert rel <= 1e-3, (name, rel)
        assert np.all(np.abs(gpu - fd) <= 1e-2 * np.abs(fd).max()), name
