"""The hand-written adjoint (rt_render_backward) against central finite
differences of the FP64 oracle at pixels away from silhouettes and shadow edges,
a closed form, replay = recompute, determinism, and the inverse-rendering loop."""
import numpy as np
import pytest
import torch

import oracle
from oracle_pins import light, mk, sphere
from paper_2305_07450_b300 import inverse, rt, scenes as S

pytestmark = pytest.mark.gpu


def small_diff_workload(W=96, H=96):
    w = S.diff_512()
    w.params.width, w.params.height = W, H
    return w


def safe_weights(w, seed=0, margin_rel=1e-3):
    """Seeded loss weights on pixels whose oracle margin exceeds 1e-3 x scene
    scale (away from silhouettes, shadow edges and light gates); zero elsewhere."""
    px = oracle.all_pixels(w.params.width, w.params.height)
    r = oracle.trace(w.scene, w.camera, w.params, px, margin=True)
    safe = r["margin"] > margin_rel * w.scene.scene_scale
    rng = np.random.default_rng(seed)
    wt = rng.normal(size=(len(px), 3)) * safe[:, None]
    return px[safe], wt[safe], wt.reshape(w.params.height, w.params.width, 3)


def oracle_loss(scene, w, px, wt):
    return float((oracle.trace(scene, w.camera, w.params, px)["rgb"] * wt).sum())


def gpu_grad(w, wimg, hitrec=True, launch=None):
    ds = rt.DeviceScene(w.scene)
    p = w.params
    hr = torch.empty(rt.hitrec_bytes(ds, p) // 4 + 1, dtype=torch.float32, device="cuda") if hitrec else None
    rt.render(ds, w.camera, p, hitrec=hr, launch=launch)
    dl = torch.zeros((p.height, p.width, 4), dtype=torch.float32, device="cuda")
    dl[..., :3] = torch.tensor(wimg, dtype=torch.float32, device="cuda")
    g = rt.render_backward(ds, w.camera, p, dl, hitrec=hr, launch=launch)
    torch.cuda.synchronize()
    assert rt.device_errors() == 0
    ds.close()
    return g.cpu().numpy().astype(np.float64)


def fd(w, px, wt, where, field, idx):
    """Central difference of the oracle loss in one FP32 record field."""
    sc = w.scene
    arr = {"sphere": sc.spheres, "plane": sc.plane, "light": sc.lights}[where]
    pos = (idx, field) if where != "plane" else (field,)
    v = float(arr[pos])
    # a step of 16 FP32 ulps: reflections off curved surfaces amplify a
    # parameter step by orders of magnitude along a path, so a step far below the
    # pixels' margins is needed for the difference to stay on one smooth branch
    h = max(16.0 * abs(float(np.spacing(np.float32(v)))), 1e-7)
    vals = []
    for sgn in (1, -1):
        new = S.Scene(spheres=sc.spheres.copy(), plane=sc.plane.copy(), lights=sc.lights.copy(), scale=sc.scale)
        a = {"sphere": new.spheres, "plane": new.plane, "light": new.lights}[where]
        a[pos] = np.float32(v + sgn * h)
        vals.append((float(a[pos]), oracle_loss(new, w, px, wt)))
    (vp, lp), (vm, lm) = vals
    return (lp - lm) / (vp - vm)


def test_adjoint_matches_oracle_finite_differences():
    w = small_diff_workload()
    px, wt, wimg = safe_weights(w)
    assert len(px) > 2000
    g = gpu_grad(w, wimg)
    N, L = w.scene.n_spheres, w.scene.n_lights
    # the spheres that matter most to this loss, every field; the plane; every light
    mag = np.abs(g[: 8 * N].reshape(N, 8)).sum(1)
    checks = []
    for i in np.argsort(-mag)[:5]:
        for f_rec, f_g in ((4, 0), (5, 1), (6, 2), (7, 3), (9, 4), (0, 5), (1, 6), (2, 7)):
            checks.append(("sphere", f_rec, int(i), 8 * int(i) + f_g))
    for f_rec, f_g in ((4, 0), (5, 1), (6, 2), (7, 3), (9, 4)):
        checks.append(("plane", f_rec, 0, 8 * N + f_g))
    for l in range(L):
        for c in range(4):
            checks.append(("light", c, l, 8 * (N + 1) + 4 * l + c))
    got = np.array([g[j] for *_, j in checks])
    want = np.array([fd(w, px, wt, where, f, i) for where, f, i, _ in checks])
    scale = np.abs(want).max()
    bad = np.abs(got - want) > 2e-3 * np.abs(want) + 2e-4 * scale
    assert not bad.any(), [(checks[k], got[k], want[k]) for k in np.nonzero(bad)[0]]


def test_adjoint_closed_form_single_sphere():
    """Depth 0, one sphere, one light: pixel = A c + S with S the same in every
    channel, so dpixel_r/dalbedo_r = A = (R - G) / (c_r - c_g)."""
    alb = (0.8, 0.3, 0.5)
    sc, cam, p = mk(spheres=[sphere((0, 0, 0), 1.0, albedo=alb)], lights=[light((3, 4, -5), 0.9)],
                    camera=(0, 0, -5, 0, 0, 60), W=32, H=32, D=0, ka=0.1)
    w = S.Workload("one_sphere", sc, cam, p)
    img = rt.render(rt.DeviceScene(sc), cam, p).cpu().numpy()
    x, y = 14, 13
    wimg = np.zeros((32, 32, 3))
    wimg[y, x, 0] = 1.0
    g = gpu_grad(w, wimg)
    A = (img[y, x, 0] - img[y, x, 1]) / (np.float32(alb[0]) - np.float32(alb[1]))
    assert abs(g[0] - A) < 1e-5 * max(1.0, abs(A)), (g[0], A)
    assert abs(g[1]) == 0 and abs(g[2]) == 0


def test_replay_equals_recompute_and_is_deterministic():
    w = small_diff_workload(64, 48)
    rng = np.random.default_rng(1)
    wimg = rng.normal(size=(48, 64, 3))
    a = gpu_grad(w, wimg, hitrec=True)
    b = gpu_grad(w, wimg, hitrec=False)
    c = gpu_grad(w, wimg, hitrec=True)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)
    # the tiled loop (geometry staged per warp chunk) gives the same paths and sums
    d = gpu_grad(w, wimg, hitrec=False, launch={"staging": 3})
    e = gpu_grad(w, wimg, hitrec=True, launch={"staging": 3})
    assert np.array_equal(a, d) and np.array_equal(a, e)


def test_autograd_function_matches_direct_call():
    w = small_diff_workload(64, 64)
    P = inverse.SceneParams(w.scene)
    ds = rt.DeviceScene(w.scene)
    img = inverse.render_image(P, ds, w.camera, w.params)
    wimg = torch.randn(img.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    (img * wimg).sum().backward()
    g = gpu_grad(w, wimg[..., :3].cpu().numpy())
    N = w.scene.n_spheres
    assert np.allclose(P.albedo.grad.cpu().numpy(), g[: 8 * N].reshape(N, 8)[:, 0:3], rtol=0, atol=0)
    assert np.allclose(P.light_pos.grad.cpu().numpy(), g[8 * (N + 1):].reshape(-1, 4)[:, 0:3], rtol=0, atol=0)


def test_inverse_rendering_reduces_loss_and_parameter_error(tmp_path):
    w = small_diff_workload(128, 128)
    truth = S.perturbed_target(w)
    tgt = inverse.target_image(truth, w)
    out = inverse.inverse_render(w, tgt, steps=100, lr=0.05, truth=truth, checkpoint=str(tmp_path / "ck.pt"),
                                 checkpoint_every=50)
    h = out["history"]
    assert h[-1] < h[0] / 5, (h[0], h[-1])
    assert out["light_rmse"][1] < out["light_rmse"][0]
    # resume from the checkpoint: continues where it stopped
    out2 = inverse.inverse_render(w, tgt, steps=110, lr=0.05, checkpoint=str(tmp_path / "ck.pt"))
    assert len(out2["history"]) == 110 and out2["history"][99] == h[99]


def test_backward_refuses_the_coupled_mode():
    w = small_diff_workload(32, 32)
    w.params.refl_coupled, w.params.max_reflectivity = 1, 64.0
    ds = rt.DeviceScene(w.scene)
    dl = torch.zeros((32, 32, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rt.RtError):
        rt.render_backward(ds, w.camera, w.params, dl)


@pytest.mark.parametrize("W,H", [(264, 200), (96, 40)])
def test_gradient_sum_over_cta_partials_in_its_stated_order(W, H):
    """The second launch sums the per-CTA partials the workspace holds in the
    order the header states (warp w: partials w, w + 32, ... in turn; then the 32
    warp sums in turn), FP32: 425 partials (full groups of eight loads and a
    ragged tail) and 18 (fewer partials than warps)."""
    w = small_diff_workload(W, H)
    ds = rt.DeviceScene(w.scene)
    p = w.params
    launch = {"block_x": 16, "block_y": 8}
    dl = torch.randn((H, W, 4), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    G = rt.grad_count(ds)
    n_parts = ((W + 15) // 16) * ((H + 7) // 8)
    ws = torch.full((n_parts * G + 64,), float("nan"), dtype=torch.float32, device="cuda")
    g = rt.render_backward(ds, w.camera, p, dl, hitrec=None, workspace=ws, launch=launch)
    torch.cuda.synchronize()
    ds.close()
    parts = ws[: n_parts * G].view(n_parts, G).cpu().numpy()
    assert np.isfinite(parts).all()
    want = np.zeros(G, np.float32)
    for wi in range(32):
        acc = np.zeros(G, np.float32)
        for b in range(wi, n_parts, 32):
            acc = acc + parts[b]
        want = want + acc
    assert np.array_equal(g.cpu().numpy(), want)
