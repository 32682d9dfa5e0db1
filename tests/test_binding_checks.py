"""The Python binding's argument checks, on the CPU: a host tensor, a tensor
on another GPU, the wrong element type, a non-contiguous or too small tensor
never reaches the library (KpError with KP_EINVAL), and well-formed
arguments pass through unchanged.  The library itself is replaced by a
recorder, so no call reaches a device."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kpsvd():
    from paper_2311_15393_gb300 import build
    build.build()
    from paper_2311_15393_gb300 import kpsvd
    return kpsvd


class CudaLike:
    """Stands in for a CUDA tensor: device, dtype, size and layout only."""

    def __init__(self, numel, dtype=torch.float32, index=0, contiguous=True, shape=None, addr=0x7000):
        self.device = torch.device("cuda", index)
        self.dtype = dtype
        self._numel, self._contiguous, self._addr = numel, contiguous, addr
        self.shape = shape or (numel,)

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        return self._addr

    def dim(self):
        return len(self.shape)


class Recorder:
    """Replaces the loaded library: records every call, returns KP_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append((name, args))
            return 0
        return f


@pytest.fixture
def rec(kpsvd, monkeypatch):
    r = Recorder()
    monkeypatch.setattr(kpsvd, "_lib", r)
    return r


def _ctx(kpsvd, vec="f32", n=8):
    ctx = kpsvd.KpContext.__new__(kpsvd.KpContext)
    ctx._h, ctx.device, ctx.n_r, ctx.n_c, ctx.vec = None, 0, n, n, vec
    return ctx


def _bad_variants(n, dtype):
    """(name, argument) pairs that must be rejected where a CUDA `dtype`
    tensor of n elements on cuda:0 is required."""
    other = torch.float64 if dtype == torch.float32 else torch.float32
    return [("host tensor", torch.zeros(n, dtype=dtype)),
            ("other GPU", CudaLike(n, dtype, index=1)),
            ("element type", CudaLike(n, other)),
            ("not contiguous", CudaLike(n, dtype, contiguous=False)),
            ("too small", CudaLike(n - 1, dtype))]


def _rejected(kpsvd, call):
    with pytest.raises(kpsvd.KpError) as e:
        call()
    assert e.value.status == kpsvd.KP_EINVAL


@pytest.mark.parametrize("vec,dt", [("f32", torch.float32), ("f64", torch.float64)])
def test_context_methods_check_every_image(kpsvd, rec, vec, dt):
    ctx = _ctx(kpsvd, vec)
    good = lambda: CudaLike(64, dt)  # noqa: E731
    calls = {
        "kp_forward": lambda a, b, c: ctx.kp_forward(a, b, 0.01, c),
        "tik_pcg": lambda a, b: ctx.tik_pcg(a, 0.1, 1e-6, 10, True, b),
        "choose_lambda": lambda a, b: ctx.choose_lambda(a, "opt", 0.0, b),
        "kp_apply_A": lambda a, b: ctx.kp_apply_A(a, b),
        "kp_apply_K": lambda a, b: ctx.kp_apply_K(a, b, 0.1),
        "kp_apply_Minv": lambda a, b: ctx.kp_apply_Minv(a, b, 0.1),
    }
    for name, call in calls.items():
        nargs = call.__code__.co_argcount
        for pos in range(nargs):
            for why, bad in _bad_variants(64, dt):
                args = [good() for _ in range(nargs)]
                args[pos] = bad
                n0 = len(rec.calls)
                _rejected(kpsvd, lambda: call(*args))
                assert len(rec.calls) == n0, (name, pos, why)    # never reached the library
        args = [CudaLike(64, dt, addr=0x1000 * (k + 1)) for k in range(nargs)]
        call(*args)
        got = rec.calls[-1]
        assert got[0] == name
        for k in range(nargs):
            assert 0x1000 * (k + 1) in got[1], (name, k)


def test_setup_and_features_check_their_buffers(kpsvd, rec):
    ctx = _ctx(kpsvd, "f32")
    for why, bad in _bad_variants(64, torch.float64):
        _rejected(kpsvd, lambda: ctx.kp_setup(bad, 8, 8, (4, 4), "zero", 1, "f32", "f32", "f32"))
    ctx.kp_setup(CudaLike(64, torch.float64, addr=0x5000), 8, 8, (4, 4), "zero", 1, "f32", "f32", "f32")
    assert rec.calls[-1][0] == "kp_setup" and rec.calls[-1][1][1] == 0x5000
    for why, bad in _bad_variants(256, torch.float32):
        _rejected(kpsvd, lambda: ctx.kp_lambda_features(CudaLike(64), bad))
    ctx.kp_lambda_features(CudaLike(64), CudaLike(256, addr=0x6000))
    assert rec.calls[-1][1][2] == 0x6000


def test_before_setup_only_the_device_is_checked(kpsvd, rec):
    """Without a problem the C call returns KP_ESTATE; the binding checks only
    that the tensors live on the context's GPU."""
    ctx = _ctx(kpsvd, "f64", n=0)
    ctx.tik_pcg(CudaLike(4, torch.float32), 0.1, 1e-6, 10, True, CudaLike(4, torch.float32))
    assert rec.calls[-1][0] == "tik_pcg"
    _rejected(kpsvd, lambda: ctx.tik_pcg(torch.zeros(4), 0.1, 1e-6, 10, True, CudaLike(4)))


def test_raw_addresses_and_none_pass_through(kpsvd, rec):
    ctx = _ctx(kpsvd, "f32")
    ctx.choose_lambda(0x9000, "gcv")
    assert rec.calls[-1][1][1] == 0x9000 and rec.calls[-1][1][4] is None


def test_batch_checks_each_problem(kpsvd, rec):
    def prob(psf=None, b=None, x=None):
        return dict(psf=CudaLike(64, torch.float64) if psf is None else psf, b=CudaLike(64) if b is None else b,
                    x=CudaLike(64) if x is None else x,
                    n_r=8, n_c=8, center=(4, 4), bc="zero", op_rank=1)
    for key, dt in (("psf", torch.float64), ("b", torch.float32), ("x", torch.float32)):
        for why, bad in _bad_variants(64, dt):
            _rejected(kpsvd, lambda: kpsvd.kp_solve_batch([prob(), prob(**{key: bad})]))
    assert not rec.calls
    kpsvd.kp_solve_batch([prob(), prob()])
    assert rec.calls[-1][0] == "kp_solve_batch"


def test_mlp_checks_its_batches(kpsvd, rec):
    m = kpsvd.Mlp.__new__(kpsvd.Mlp)
    m._h, m.device, m.param_count = None, 0, 10
    X = lambda n=5: CudaLike(n * kpsvd.N_FEAT, shape=(n, kpsvd.N_FEAT))  # noqa: E731
    _rejected(kpsvd, lambda: m.forward(CudaLike(5 * 255, shape=(5, 255)), CudaLike(5)))     # feature width
    _rejected(kpsvd, lambda: m.forward(torch.zeros(5, kpsvd.N_FEAT), CudaLike(5)))           # host tensor
    for why, bad in _bad_variants(5, torch.float32):
        _rejected(kpsvd, lambda: m.forward(X(), bad))
        _rejected(kpsvd, lambda: m.train_step(X(), bad, 1e-3))
    assert not rec.calls
    m.forward(X(), CudaLike(5))
    m.train_step(X(), CudaLike(5), 1e-3)
    assert [c[0] for c in rec.calls] == ["kp_mlp_forward", "kp_mlp_train_step"]
    assert rec.calls[0][1][2] == 5      # batch size from X


def test_noalloc_checks_factor_and_image_sizes(kpsvd, rec, monkeypatch):
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    f32, f64 = torch.float32, torch.float64
    args = lambda **kw: dict(dict(Vc=CudaLike(64), Vr=CudaLike(36), sigma=CudaLike(48, f64),  # noqa: E731
                                  r=CudaLike(48), z=CudaLike(48)), **kw)
    for key, n, dt in (("Vc", 64, f32), ("Vr", 36, f32), ("sigma", 48, f64), ("r", 48, f32), ("z", 48, f32)):
        for why, bad in _bad_variants(n, dt):
            a = args(**{key: bad})
            _rejected(kpsvd, lambda: kpsvd.kp_apply_Minv_noalloc(a["Vc"], a["Vr"], a["sigma"], 8, 6, 0.1,
                                                                 a["r"], a["z"], stream=0))
    assert not rec.calls
    a = args()
    kpsvd.kp_apply_Minv_noalloc(a["Vc"], a["Vr"], a["sigma"], 8, 6, 0.1, a["r"], a["z"], stream=0)
    assert rec.calls[-1][0] == "kp_apply_Minv_noalloc"
