"""The load-balancing fine-tune (Sec. 4.4 total loss) on a 200k-Gaussian
clustered scene at 480x270.  Without the load term the image loss falls and the training views fit
their targets better.  With lambda_load = 0.45 the load gradient's reading
decides the outcome: under the early-stop reading the load spreads less than
without the load term (lower std of l_i on the training views), which is the
paper's aim; the straight-through reading is run and reported (it can raise
the spread: lowering alpha delays the early stop)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_finetune_fits_targets_and_load_term_balances():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_08669_gb300 import scenes as S
    from paper_2409_08669_gb300.finetune import FinetuneConfig, Finetuner, evaluate, render_targets
    from paper_2409_08669_gb300.raster import Rasterizer, upload
    base = S.cluster_scene(n=200_000, seed=1)
    target = S.perturbed_scene(base, seed=4)
    cams = S.orbit_cameras(8, width=480, height=270)
    st = S.Settings(mode=S.MODE_AABB)
    st_stop = S.Settings(mode=S.MODE_AABB, load_grad=S.LOAD_GRAD_TERMINATION)
    rast = Rasterizer(max_gaussians=base.n, pair_capacity=1 << 25, max_width=480, max_height=270)
    try:
        tgt = render_targets(rast, upload(target), cams, st)
        before = evaluate(rast, upload(base), cams, tgt, st, repeats=1)
        res = {}
        for name, cfg, s in (("plain", FinetuneConfig(steps=150, lambda_l1=0.8, lambda_ssim=0.2,
                                                      lambda_load=0.0), st),
                             ("straight", FinetuneConfig(steps=150), st),
                             ("stop", FinetuneConfig(steps=150), st_stop)):
            ft = Finetuner(base, cams, tgt, rast, s, cfg)
            first = float(ft.step())
            for _ in range(cfg.steps - 1):
                last = ft.step()
            torch.cuda.synchronize()
            res[name] = evaluate(rast, ft.activated_copy(), cams, tgt, st, repeats=1)
            res[name]["first_loss"], res[name]["last_loss"] = first, float(last)
    finally:
        rast.close()
    print(before, res)
    assert res["plain"]["last_loss"] < res["plain"]["first_loss"]
    assert res["plain"]["psnr_db"] > before["psnr_db"] + 1.0
    assert res["stop"]["psnr_db"] > before["psnr_db"]
    assert res["stop"]["load_std"] < 0.95 * res["plain"]["load_std"]   # measured: 15.9 vs 18.6
