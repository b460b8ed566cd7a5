"""The FP32 wavefront kernel families (one-row, two-row, register at every depth) give
bitwise the same states and residual reports as the single-sweep streaming
kernel, which the oracle tests pin; each family is selected on a context of
its own through the PX_OPT_FP32_FAMILY option."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FAMILIES = {"default": 0, "w1": 1, "w2": 2, "r": 3, "rp": 4}


@pytest.mark.parametrize("family", ["w1", "w2", "r", "rp", "default"])
def test_family_bitwise_equals_single_sweep(family):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_FP32_FAMILY, FAMILIES[family])
        assert ctx.get_option(px.PX_OPT_FP32_FAMILY) == FAMILIES[family]
        g = torch.Generator(device="cuda")
        g.manual_seed(7)
        for (nx, ny) in [(1000, 1000), (260, 150), (16, 8), (4, 4), (12, 37), (252, 40),
                         (256, 33), (2052, 300), (124, 64)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            o1, ot = torch.empty_like(phi), torch.empty_like(phi)
            r1 = torch.zeros(11, dtype=torch.float64, device="cuda")
            rt = torch.zeros_like(r1)
            px.relax_n(phi, o1, rho, h, 2 / 3, 11, 1, r1, 1, ctx=ctx)
            for tb in range(2, 9):
                px.relax_n(phi, ot, rho, h, 2 / 3, 11, tb, rt, 1, ctx=ctx)
                torch.cuda.synchronize()
                assert torch.equal(o1, ot) and torch.equal(r1, rt), (family, nx, ny, tb)
    finally:
        ctx.close()


def test_option_values_are_checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        for opt, bad in ((px.PX_OPT_FP32_FAMILY, 5), (px.PX_OPT_FP32_FAMILY, -1),
                         (px.PX_OPT_RB_SWEEPS_PER_LAUNCH, 5), (px.PX_OPT_BATCH_LAUNCHES, 2),
                         (px.PX_OPT_BATCH_LAUNCHES, -1), (px.PX_OPT_RB_FP64_PASSES, 3),
                         (px.PX_OPT_MG_PROLONG, 2),
                         (99, 0)):
            with pytest.raises(px.PxError) as ei:
                ctx.set_option(opt, bad)
            assert ei.value.status == px.PX_EINVAL
    finally:
        ctx.close()


def test_balanced_register_kernel_bitwise():
    """On fields large enough for the register wavefront (2^23 cells or more),
    where warps rebalance their rows at run time, depths 3 to 8 give bitwise
    the states and reports of the single-sweep kernel, launch after launch
    (the balance words are reused)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for (nx, ny) in [(4096, 4096), (4100, 4097), (8192, 2052), (2900, 2896)]:
        h = 1.0 / nx
        rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
        phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
        a, b = torch.empty_like(phi), torch.empty_like(phi)
        ra = torch.zeros(8, dtype=torch.float64, device="cuda")
        rb = torch.zeros_like(ra)
        px.relax_n(phi, b, rho, h, 2 / 3, 8, 1, rb, 1)
        for tb in (8, 3, 4, 5, 6, 7, 8):
            px.relax_n(phi, a, rho, h, 2 / 3, 8, tb, ra, 1)
            torch.cuda.synchronize()
            assert torch.equal(a, b) and torch.equal(ra, rb), (nx, ny, tb)


@pytest.mark.parametrize("family", ["r", "rp"])
def test_register_kernel_report_spacings_bitwise(family):
    """The register wavefront reports only the stages whose input state is
    due (a flag per stage); for report spacings 1, 2, 3, 5, 16 and no report,
    its states and reports are bitwise those of the single-sweep kernel, at
    every depth 2..8 (8-warp and 12-warp launches) and sizes with several
    strips and ranges."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_FP32_FAMILY, FAMILIES[family])
        g = torch.Generator(device="cuda")
        g.manual_seed(23)
        for (nx, ny) in [(1000, 1002), (2052, 300), (124, 64)]:
            h = 1.0 / nx
            rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
            o1, ot = torch.empty_like(phi), torch.empty_like(phi)
            for every in (1, 2, 3, 5, 16, 0):
                n = 17
                k = (n + every - 1) // every if every else 1
                r1 = torch.zeros(k, dtype=torch.float64, device="cuda")
                rt = torch.full_like(r1, -1.0)
                px.relax_n(phi, o1, rho, h, 2 / 3, n, 1, r1 if every else None, every, ctx=ctx)
                for tb in range(2, 9):
                    rt.fill_(-1.0)
                    px.relax_n(phi, ot, rho, h, 2 / 3, n, tb, rt if every else None, every,
                               ctx=ctx)
                    torch.cuda.synchronize()
                    assert torch.equal(o1, ot), (family, nx, ny, tb, every)
                    if every:
                        assert torch.equal(r1, rt), (family, nx, ny, tb, every)
    finally:
        ctx.close()


@pytest.mark.parametrize("sweeps", [2, 4])
def test_red_black_register_report_spacings_bitwise(sweeps):
    """Red-black register wavefront launches with reports on every sweep,
    every other or third sweep and none give bitwise the states and reports
    of the two-pass kernels (pitched copies take those)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2307_07931_b300 as px
    ctx = px.Context(torch.cuda.current_device())
    try:
        ctx.set_option(px.PX_OPT_RB_SWEEPS_PER_LAUNCH, sweeps)
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        nx, ny = 1000, 1002
        h = 1.0 / nx
        rho = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)
        phi = torch.randn(ny, nx, device="cuda", dtype=torch.float32, generator=g)

        def pitched(a):
            b = torch.zeros(ny, nx + 1, device="cuda", dtype=torch.float32)[:, :nx]
            b.copy_(a)
            return b
        pp, rp, op = pitched(phi), pitched(rho), pitched(torch.zeros_like(phi))
        out = torch.empty_like(phi)
        for every in (1, 2, 3, 0):
            n = 13
            k = (n + every - 1) // every if every else 1
            r1 = torch.zeros(k, dtype=torch.float64, device="cuda")
            r2 = torch.full_like(r1, -1.0)
            px.rbsor_n(pp, op, rp, h, 1.3, n, r1 if every else None, every, ctx=ctx)
            px.rbsor_n(phi, out, rho, h, 1.3, n, r2 if every else None, every, ctx=ctx)
            torch.cuda.synchronize()
            assert torch.equal(op, out), every
            if every:
                assert torch.equal(r1, r2), every
    finally:
        ctx.close()
