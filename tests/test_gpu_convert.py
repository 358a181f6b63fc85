"""The refinement residual stores x * 2^e as FP32 with an integer-pipe
round-to-nearest-even conversion (ps_op_scale_to_fp32).  It must give, bit for
bit, what CUDA's own double -> float conversion gives for the exactly scaled
double: normal results, exact ties (both parities), results in the FP32
subnormal range, the smallest normal reached by rounding, overflow to
infinity, signed zeros."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_03563_gb300 as P
    P.capi.lib()
    from paper_2605_03563_gb300 import ops as O
    return O


def _cases(rng):
    vals = []
    # random doubles over a wide exponent range, both signs
    m = rng.uniform(1.0, 2.0, 20000) * rng.choice([-1.0, 1.0], 20000)
    vals.append(np.ldexp(m, rng.integers(-160, 160, 20000)))
    # exact ties and their neighbours: f + ulp(f)/2 (+-1 double ulp)
    f = rng.uniform(1.0, 2.0, 4000).astype(np.float32).astype(np.float64)
    f = np.ldexp(f, rng.integers(-140, 128, 4000))
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    t = f + ulp / 2
    vals += [t, np.nextafter(t, np.inf), np.nextafter(t, -np.inf), -t]
    # around the FP32 subnormal range and the smallest normal
    tiny = np.ldexp(rng.uniform(0.0, 2.0, 4000), rng.integers(-152, -124, 4000))
    vals += [tiny, -tiny, np.array([2.0 ** -126 * (1 - 2.0 ** -25), 2.0 ** -150, 2.0 ** -150 * 1.0000001,
                                    2.0 ** -151, 2.0 ** -149 * 1.5, 2.0 ** -149 * 2.5])]
    # around the largest finite FP32 value
    fm = float(np.finfo(np.float32).max)
    vals.append(np.array([fm, fm * (1 + 2.0 ** -25), fm * (1 + 2.0 ** -24), fm * 2, 3.5e38, -3.5e38]))
    vals.append(np.array([0.0, -0.0, 1.0, -1.0, 0.5, 3.0]))
    return np.concatenate(vals)


@pytest.mark.parametrize("e", [0, 1, -1, 37, -37, 100, -100])
def test_scale_to_fp32_matches_cuda_conversion(ops, e):
    rng = np.random.default_rng(100 + e)
    base = _cases(rng)
    # inputs x such that x * 2^e is the case value (exact in FP64)
    x = torch.from_numpy(np.ldexp(base, -e)).cuda()
    out = torch.empty(x.numel(), dtype=torch.float32, device="cuda")
    ops.scale_to_fp32(x, e, out)
    ref = (x * (2.0 ** e)).to(torch.float32)
    torch.cuda.synchronize()
    a, b = out.view(torch.int32).cpu().numpy(), ref.view(torch.int32).cpu().numpy()
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, [(float(x[i]), int(a[i]), int(b[i])) for i in bad[:5]]


def test_scale_to_fp32_rejects_large_exponent(ops):
    import paper_2605_03563_gb300 as P
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    with pytest.raises(P.capi.PoissonError):
        ops.scale_to_fp32(x, 101, out)


@pytest.mark.parametrize("p", [0, 3, -3, 64, -64, 100, -100])
def test_add_scaled_fp32_matches_fma(ops, p):
    """The refinement's correction phi += e * 2^p builds e * 2^p from e's FP32
    encoding on the integer pipe and adds once: bit for bit what CUDA's
    conversion and FMA give, for FP32 normals, subnormals, signed zeros and
    infinities, against FP64 addends of every magnitude (cancellation, ties)."""
    rng = np.random.default_rng(300 + p)
    n = 40000
    f = (rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n) * np.ldexp(1.0, rng.integers(-149, 128, n)))
    f = f.astype(np.float32)
    sub = np.ldexp(rng.integers(1, 1 << 23, 2000).astype(np.float64), -149).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, np.finfo(np.float32).max,
                        np.finfo(np.float32).tiny, 2.0 ** -149], dtype=np.float32)
    e = np.concatenate([f, sub, -sub, special])
    m = e.size
    base = np.ldexp(rng.uniform(-2.0, 2.0, m), rng.integers(-300, 300, m))
    # addends that cancel the correction to a few bits, and exact ties
    close = -np.ldexp(e.astype(np.float64), p)
    fin = np.isfinite(close)
    base[: m // 4][fin[: m // 4]] = close[: m // 4][fin[: m // 4]] * (1 + 2.0 ** -30)
    e_t = torch.from_numpy(e).cuda()
    phi = torch.from_numpy(base).cuda()
    ref = torch.addcmul(phi, e_t.double(), torch.full_like(phi, 2.0 ** p))
    got = phi.clone()
    ops.add_scaled_fp32(e_t, p, got)
    torch.cuda.synchronize()
    a, b = got.view(torch.int64).cpu().numpy(), ref.view(torch.int64).cpu().numpy()
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, [(float(e[i]), float(base[i]), int(a[i]), int(b[i])) for i in bad[:5]]


def test_add_scaled_fp32_rejects_large_exponent(ops):
    import paper_2605_03563_gb300 as P
    e = torch.zeros(4, dtype=torch.float32, device="cuda")
    phi = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(P.capi.PoissonError):
        ops.add_scaled_fp32(e, -101, phi)
