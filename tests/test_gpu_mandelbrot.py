"""The Mandelbrot kernel and actor stage (Sec. 5.4) against the oracle, bit
for bit: the paper's rectangle at small and full size (1920 x 1080, 100
steps; sampled rows of 16000 x 16000 at 1000 steps), the whole set, and the
actor stage with its image read back (value mode)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_util import empty, stream, to_host  # noqa: E402

REGION = oracle.MANDELBROT_REGION


@pytest.fixture(scope="module")
def ka(cuda_ok):
    import paper_1709_07781_gb300 as m
    return m


def gpu_image(ka, w, h, region, iters):
    out = empty(w * h)
    assert ka.ka_mandelbrot(out, w, h, *region, iters, stream()) == 0
    torch.cuda.synchronize()
    return to_host(out, w * h).reshape(h, w)


@pytest.mark.parametrize("w,h,region,iters", [
    (1, 1, REGION, 100), (37, 23, REGION, 100), (320, 180, REGION, 100), (64, 64, REGION, 1000),
    (200, 150, (-2.0, -1.25, 0.5, 1.25), 256), (33, 17, (-0.75, 0.05, -0.74, 0.06), 5000),
    # step limits of 0 to 3 and odd ones: every exit of the kernel's two-step loop
    (48, 32, (-2.0, -1.25, 0.5, 1.25), 0), (48, 32, (-2.0, -1.25, 0.5, 1.25), 1),
    (48, 32, (-2.0, -1.25, 0.5, 1.25), 2), (48, 32, (-2.0, -1.25, 0.5, 1.25), 3),
    (48, 32, (-2.0, -1.25, 0.5, 1.25), 7), (64, 48, REGION, 101)])
def test_mandelbrot_matches_oracle(ka, w, h, region, iters):
    assert np.array_equal(gpu_image(ka, w, h, region, iters), oracle.mandelbrot(w, h, *region, iters))


def test_mandelbrot_full_hd_and_sampled_large(ka):
    img = gpu_image(ka, 1920, 1080, REGION, 100)
    assert np.array_equal(img, oracle.mandelbrot(1920, 1080, *REGION, 100))
    W = H = 16000
    out = torch.empty(W * H, dtype=torch.int32, device="cuda")
    assert ka.ka_mandelbrot(out, W, H, *REGION, 1000, stream()) == 0
    torch.cuda.synchronize()
    re_min, im_min, re_max, im_max = (np.float32(v) for v in REGION)
    dim = np.float32(np.float32(im_max - im_min) / np.float32(H))
    for y in (0, 1, 4321, 9999, H - 1):
        # the row's imaginary part, made by the same two single-precision operations
        ci = float(np.float32(im_min + np.float32(np.float32(y) * dim)))
        row = oracle.mandelbrot(W, 1, float(re_min), ci, float(re_max), ci + 1.0, 1000)[0]
        got = out[y * W:(y + 1) * W].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, row), y


def test_mandelbrot_actor_stage(ka):
    s, sysh = ka.ka_system_create(0)
    assert s == 0
    try:
        s, a = ka.ka_spawn_stage(sysh, ka.KA_STAGE_MANDELBROT, 192, 100, 108)
        assert s == 0, ka.ka_strerror(s)
        out = np.zeros(192 * 108, dtype=np.uint32)
        s, req = ka.ka_request(a, ka.make_msg(h_out=out))
        assert s == 0
        s, msg = ka.ka_receive(req)
        assert s == 0 and msg.count == 192 * 108
        assert np.array_equal(out.reshape(108, 192), oracle.mandelbrot(192, 108, *REGION, 100))
        for i in range(msg.n_refs):
            ka.ka_ref_release(msg.refs[i])
        ka.ka_actor_release(a)
        # invalid sizes are refused at spawn
        assert ka.ka_spawn_stage(sysh, ka.KA_STAGE_MANDELBROT, 0, 100, 10)[0] == ka.KA_E_ARG
        assert ka.ka_spawn_stage(sysh, ka.KA_STAGE_MANDELBROT, 70000, 100, 70000)[0] == ka.KA_E_ARG
    finally:
        ka.ka_system_destroy(sysh, 1)
