"""CPU replay of the planned GPU passes (tests/emu): every access in bounds, no
stale or colliding shared-memory slot, every output written once, and the
replayed arithmetic within the FP32 tolerance of the FP64 oracle.  This checks
the kernels' index logic before they run; the GPU parity tests are separate."""
import numpy as np
import pytest

from emu import emu
from paper_1505_08067_gb300 import synth


def _check(oracle, shape, batch, direction=-1, seed=5, specialised=True, **opts):
    n = int(np.prod(shape))
    x = synth.uniform(seed, batch, n).reshape((batch,) + tuple(shape))
    y, nerr, msg = emu.run(x, shape, direction=direction, specialised=specialised, **opts)
    assert nerr == 0, msg
    if batch == 0:
        return
    ref = oracle.fft(x, direction) if len(shape) == 1 else oracle.fft2d(x, direction)
    err = oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))
    tol = 1e-6 * max(1.0, np.log2(n))
    assert np.max(err) <= tol, (shape, batch, opts, np.max(err))


@pytest.mark.parametrize("logn", range(0, 15))
@pytest.mark.parametrize("batch", [1, 3])
@pytest.mark.parametrize("direction", [-1, 1])
def test_single_pass(oracle, logn, batch, direction):
    _check(oracle, (2 ** logn,), batch, direction)


@pytest.mark.parametrize("logn", range(8, 15))
@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("specialised", [True, False])
def test_compile_time_shapes(oracle, logn, direction, specialised):
    """The batch sizes the benchmark uses select the compile-time kernels; the
    generic kernel must agree on the same plan."""
    n = 2 ** logn
    batch = 2 ** 16 // n
    st = {}
    x = synth.uniform(9, batch, n)
    y, nerr, msg = emu.run(x, (n,), direction=direction, specialised=specialised, stats=st)
    assert nerr == 0, msg
    expect_staged = specialised and logn >= 13      # staged kernel for 2^13, 2^14 (2^12: register)
    assert st["staged_passes"] == (1 if expect_staged else 0)
    assert st["special_passes"] == (1 if specialised and not expect_staged else 0)
    assert np.max(oracle.rel_l2(y, oracle.fft(x, direction))) <= 1e-6 * logn


@pytest.mark.parametrize("direction", [-1, 1])
def test_staged_4096_on_request(oracle, direction):
    """Variant 2 runs contiguous 4096-point transforms on the staged kernel
    (the library's own choice there is the register kernel)."""
    st = {}
    x = synth.uniform(10, 7, 4096)
    y, nerr, msg = emu.run(x, (4096,), direction=direction, stats=st, variant=2)
    assert nerr == 0, msg
    assert st["staged_passes"] == 1
    assert np.max(oracle.rel_l2(y, oracle.fft(x, direction))) <= 1e-6 * 12


@pytest.mark.parametrize("logn,batch", [(15, 2), (16, 1), (17, 1), (18, 1)])
def test_four_step(oracle, logn, batch):
    _check(oracle, (2 ** logn,), batch)
    _check(oracle, (2 ** logn,), batch, +1)


@pytest.mark.parametrize("logn,bmax", [(6, 3), (7, 4), (9, 5), (12, 6), (16, 8), (14, 7)])
def test_forced_splits(oracle, logn, bmax):
    _check(oracle, (2 ** logn,), 3, max_block_log2=bmax)


@pytest.mark.parametrize("radix,schedule", [(8, 0), (4, 0), (2, 0), (16, 0x2422), (16, 0x4222),
                                            (16, 0x1144), (16, 0x4411), (8, 0x1333)])
def test_forced_schedules_n1024(oracle, radix, schedule):
    _check(oracle, (1024,), 5, radix=radix, schedule=schedule)


@pytest.mark.parametrize("tile", [1, 2, 8, 32])
def test_tiles_with_ragged_batch(oracle, tile):
    _check(oracle, (256,), 37, tile=tile)


@pytest.mark.parametrize("shape", [(8, 16), (16, 8), (1, 64), (64, 1), (1, 1), (32, 32),
                                   (256, 512), (2 ** 14, 2)])
def test_2d(oracle, shape):
    _check(oracle, shape, 2)
    _check(oracle, shape, 1, +1)


def test_empty_batch(oracle):
    _check(oracle, (64,), 0)


def test_largest_four_step_slice(oracle):
    """The widest tile shapes of the 2^24 plan on a cheaper 2^20 replay."""
    _check(oracle, (2 ** 20,), 1)


@pytest.mark.parametrize("epilogue", [1, 2, 3, 4])
@pytest.mark.parametrize("logn", [15, 20])
def test_four_step_twiddle_sources(oracle, epilogue, logn):
    """Two-level tables, the full table and the in-kernel rotor give the same
    transform (the host replay evaluates the rotor in FP64)."""
    _check(oracle, (2 ** logn,), 1, epilogue=epilogue)
    _check(oracle, (2 ** logn,), 1, +1, epilogue=epilogue)


# tensor-core class: tolerance per precision (see test_tc_gpu.py for the reading)
TC_TOL = {1: lambda n: 2e-3, 2: lambda n: 5e-3, 3: lambda n: 5e-6 * np.log2(n)}
# six-step plans round the data at the stages of both passes (up to six):
# plain BF16 at about 2e-3 per rounded stage in quadrature needs 7e-3
SIX_STEP_TOL = {1: lambda n: 2e-3, 2: lambda n: 7e-3, 3: lambda n: 5e-6 * np.log2(n)}


@pytest.mark.parametrize("n", [16, 256, 4096])
@pytest.mark.parametrize("precision", [1, 2, 3])
def test_tensor_core_class_replay(oracle, n, precision):
    """Fragment layouts, addressing and ping-pong buffers of the warp-level
    tensor-core kernel (variant 1), with the warp MMA emulated from its
    documented fragment layout."""
    batch = 4096 // n * 2 + 1                       # two full tiles and a ragged one
    x = synth.uniform(77, batch, n)
    for d in (-1, 1):
        y, nerr, msg = emu.run(x, (n,), direction=d, precision=precision, variant=1)
        assert nerr == 0, msg
        assert np.max(oracle.rel_l2(y, oracle.fft(x, d))) <= TC_TOL[precision](n)


@pytest.mark.parametrize("logn", range(4, 15))
@pytest.mark.parametrize("precision", [1, 2, 3])
def test_tcgen05_class_replay(oracle, logn, precision):
    """The tcgen05 tensor-core kernel's loader (with the radix-2/4/8 first
    stage where N is not a power of 16), A-operand layout, row permutations,
    tensor-memory row ownership and epilogue, with the UMMA emulated from the
    operand layout the hardware reads: every A word written once per phase,
    every output once, and the transform within the class tolerance."""
    n = 2 ** logn
    tile = max(n, 4096)
    batch = tile // n * 2 + 1 if n < 4096 else 3     # two full tiles and a ragged one
    x = synth.uniform(78 + logn, batch, n)
    for d in (-1, 1):
        y, nerr, msg = emu.run(x, (n,), direction=d, precision=precision)
        assert nerr == 0, msg
        assert np.max(oracle.rel_l2(y, oracle.fft(x, d))) <= TC_TOL[precision](n), logn


@pytest.mark.parametrize("logn,precision", [(15, 1), (16, 3), (17, 2), (18, 1)])
def test_tcgen05_six_step_replay(oracle, logn, precision):
    """Tensor-core plans above 2^14 (transposes, tensor-core rows of N1 and
    N2, the six-step twiddle in the middle transpose), replayed on the CPU with
    the UMMA emulated, against the oracle, forward and inverse, batch 2."""
    n = 2 ** logn
    x = synth.uniform(90 + logn, 2, n)
    for d in (-1, 1):
        y, nerr, msg = emu.run(x, (n,), direction=d, precision=precision)
        assert nerr == 0, msg
        err = np.max(oracle.rel_l2(y, oracle.fft(x, d)))
        assert err <= SIX_STEP_TOL[precision](n), (logn, d, err)


# ---------------------------------------------------------------- convolution --

def _conv_filters(oracle, shape, batch, per_line, seed):
    """Filter spectra (complex64, the oracle's FP64 DFT of seeded kernels) in
    the layout fft_filter_t describes, and the matching oracle arguments."""
    if len(shape) == 1:
        n = shape[0]
        c = synth.uniform(seed, batch if per_line[0] else 1, n)
        h = oracle.fft(c).astype(np.complex64)
        h = h if per_line[0] else h[0]
        return [(h, batch if per_line[0] else 1, 1.0 / n)]
    rows, cols = shape
    cr = synth.uniform(seed, rows if per_line[1] else 1, cols)
    hr = oracle.fft(cr).astype(np.complex64)
    hr = hr if per_line[1] else hr[0]
    ca = synth.uniform(seed + 1, cols if per_line[0] else 1, rows)   # one kernel per column
    ha = oracle.fft(ca).astype(np.complex64)
    ha = np.ascontiguousarray(ha.T) if per_line[0] else ha[0]      # column c's filter in column c
    return [(ha, cols if per_line[0] else 1, 1.0 / rows), (hr, rows if per_line[1] else 1, 1.0 / cols)]


def conv_reference(oracle, x, shape, filters):
    if len(shape) == 1:
        h, _, sc = filters[0]
        return oracle.conv(x, h.astype(np.complex128), sc)
    (ha, _, sa), (hr, _, sr) = filters
    return oracle.conv2d(x, hr.astype(np.complex128), sr, ha.astype(np.complex128), sa)


def _check_conv(oracle, shape, batch, per_line=(False, False), seed=3, specialised=True,
                expect_special=None, **opts):
    n = int(np.prod(shape))
    x = synth.uniform(seed, batch, n).reshape((batch,) + tuple(shape))
    filters = _conv_filters(oracle, shape, batch, per_line, seed + 10)
    st = opts.pop("stats", {})
    y, nerr, msg = emu.run_conv(x, shape, filters, specialised=specialised, stats=st, **opts)
    assert nerr == 0, msg
    if expect_special is not None:
        assert st["special_passes"] == expect_special
    ref = conv_reference(oracle, x, shape, filters)
    err = oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))
    # two transforms per line (forward, inverse): twice the single-FFT bound
    tol = 2e-6 * max(1.0, np.log2(max(shape)))
    assert np.max(err) <= tol, (shape, batch, per_line, np.max(err))


@pytest.mark.parametrize("logn", range(1, 15))
@pytest.mark.parametrize("per_line", [False, True])
def test_conv_lines(oracle, logn, per_line):
    _check_conv(oracle, (2 ** logn,), 3, (per_line, False))


@pytest.mark.parametrize("logn", [12, 13, 14])
@pytest.mark.parametrize("per_line", [False, True])
def test_conv_compile_time_shapes(oracle, logn, per_line):
    """Lines of 2^12..2^14 run the staged convolution kernel (no exchange
    between the two rounds); the register kernel (variant 1) and the generic
    kernel must agree on the same plan."""
    st = {}
    _check_conv(oracle, (2 ** logn,), 3, (per_line, False), stats=st)
    assert st["staged_passes"] == 1 and st["special_passes"] == 0
    _check_conv(oracle, (2 ** logn,), 3, (per_line, False), expect_special=1, variant=1)
    _check_conv(oracle, (2 ** logn,), 3, (per_line, False), specialised=False, expect_special=0)


@pytest.mark.parametrize("shape", [(2, 2), (8, 16), (16, 8), (64, 32), (4, 8192)])
@pytest.mark.parametrize("per_line", [(False, False), (True, True), (True, False)])
def test_conv_frames(oracle, shape, per_line):
    _check_conv(oracle, shape, 2, per_line)


@pytest.mark.parametrize("cols", [8, 16])
def test_conv_azimuth_shape(oracle, cols):
    """4096-point columns (4 per tile) with one filter per column run the
    staged column kernel: each tile's filters are copied into the staging
    buffer by tensor-map boxes once its data has been read.  With one shared
    filter, or with variant 1, they run the compile-time register
    convolution kernel."""
    st = {}
    _check_conv(oracle, (4096, cols), 2, (True, False), stats=st, expect_special=0)
    assert st["staged_passes"] == 1
    st = {}
    _check_conv(oracle, (4096, cols), 2, (False, False), stats=st, expect_special=1)
    assert st["staged_passes"] == 0
    st = {}
    _check_conv(oracle, (4096, cols), 2, (True, False), stats=st, expect_special=1, variant=1)
    assert st["staged_passes"] == 0


@pytest.mark.parametrize("radix,tile", [(4, 0), (8, 2), (2, 4), (16, 8)])
def test_conv_forced_radix_and_tile(oracle, radix, tile):
    _check_conv(oracle, (1024,), 7, (True, False), radix=radix, tile=tile)


@pytest.mark.parametrize("logn,split,epilogue", [(15, 10, 2), (15, 10, 3), (16, 11, 2), (16, 11, 3),
                                                 (17, 12, 2), (17, 12, 3), (20, 10, 2), (22, 11, 3),
                                                 (22, 10, 3), (15, 10, 4), (16, 11, 4), (17, 12, 4),
                                                 (22, 11, 4)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_staged_column_first_pass(oracle, logn, split, epilogue, direction):
    """Four-step first passes of 1024 / 2048 / 4096 points run the staged
    column kernel (G = 8 / 4 / 4 columns per tile, the four-step twiddle on
    store); second passes of 1024 / 2048 / 4096 points the staged transposing
    kernel (G contiguous rows in, G columns out); the register kernels must
    agree."""
    n = 2 ** logn
    x = synth.uniform(40 + logn, 3, n)
    ref = oracle.fft(x, direction)
    for variant, staged in ((0, 2 if logn - split in (10, 11, 12) else 1), (1, 0)):
        st = {}
        y, nerr, msg = emu.run(x, (n,), direction=direction, stats=st, split_log2=split,
                               epilogue=epilogue, variant=variant)
        assert nerr == 0, msg
        assert st["staged_passes"] == staged
        assert np.max(oracle.rel_l2(y, ref)) <= 1e-6 * logn


@pytest.mark.parametrize("shape", [(4096, 8), (4096, 16)])
def test_staged_column_2d(oracle, shape):
    st = {}
    x = synth.uniform(77, 2, shape[0] * shape[1]).reshape(2, *shape)
    for d in (-1, 1):
        y, nerr, msg = emu.run(x, shape, direction=d, stats=st)
        assert nerr == 0, msg
        assert st["staged_passes"] == 1
        err = oracle.rel_l2(y.reshape(2, -1), oracle.fft2d(x, d).reshape(2, -1))
        assert np.max(err) <= 1e-6 * np.log2(x[0].size)
