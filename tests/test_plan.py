"""Host-only planning of filter-bank layouts (mf_prf_plan: no GPU needed).

The factored numerator needs separable footprints and groups trajectories
that share v_x; these tests check the planner's choices and its limits."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def mf():
    import paper_2209_09848_gb300 as m
    m.load()
    return m


def _grid(nx, ny, lo=-0.1, hi=0.1):
    from paper_2209_09848_gb300 import synth
    return synth.velocity_grid(nx, ny, lo, hi)


def test_paper_grid_plans_factored(mf):
    vx, vy = _grid(10, 10)
    info = mf.prf_plan(vx, vy, 1000)
    assert info["kernel"] == 2
    kt, th, tw = info["warps_per_group"], info["tile_h"], info["tile_w"]
    assert kt * (th // 32) * (tw // 32) <= 20 and th % 32 == 0 and tw in (32, 64)
    # groups never mix v_x: each of the 10 columns of the grid splits on its own
    assert info["groups"] == 10 * -(-10 // kt)
    assert info["window_rows"] <= 256 and info["smem_bytes"] <= 227 * 1024
    assert 2 <= info["stages"] <= 6


def test_general_kernel_on_request(mf):
    vx, vy = _grid(10, 10)
    info = mf.prf_plan(vx, vy, 1000, kernel=1)
    assert info["kernel"] == 1 and info["warps_per_group"] in (16, 8, 4, 2)
    info = mf.prf_plan(vx, vy, 1000, shape=2)
    assert info["kernel"] == 1 and info["warps_per_group"] == 4


def test_distinct_vx_gives_single_trajectory_groups(mf):
    g = np.random.default_rng(3)
    vx = g.uniform(-0.1, 0.1, 40)
    vy = g.uniform(-0.1, 0.1, 40)
    info = mf.prf_plan(vx, vy, 500)
    assert info["kernel"] == 2 and info["groups"] == 40  # one trajectory per CTA


def test_forced_geometry_is_reported(mf):
    vx, vy = _grid(10, 10)
    info = mf.prf_plan(vx, vy, 1000, kernel=2, group=4, tile_h=128, tile_w=32, stages=3, segments=1)
    assert (info["warps_per_group"], info["tile_h"], info["tile_w"], info["stages"]) == (4, 128, 32, 3)
    assert info["time_segments"] == 1
    assert info["groups"] == 30
    # rows: tile + footprint + the largest s_y spread of a group; the 10 v_y
    # of a column split into groups of 4, 3 and 3 consecutive values
    gy = np.linspace(-0.1, 0.1, 10)
    s_last = np.floor(gy * 999 + 0.5)
    spread = max(s_last[j - 1] - s_last[i] for i, j in ((0, 4), (4, 7), (7, 10)))
    assert info["window_rows"] == 128 + 4 + spread


@pytest.mark.parametrize("opts", [dict(kernel=3), dict(kernel=2, group=21), dict(kernel=2, tile_h=48),
                                  dict(kernel=2, tile_w=96), dict(kernel=2, stages=1), dict(kernel=2, stages=7),
                                  dict(kernel=2, segments=17), dict(kernel=2, segments=-1)])
def test_invalid_layout_options(mf, opts):
    vx, vy = _grid(3, 3)
    with pytest.raises(mf.MFError) as e:
        mf.prf_plan(vx, vy, 10, **opts)
    assert e.value.status == 1


def test_window_too_tall_is_unsupported(mf):
    # 10 v_y spanning 2 px/frame over 140 frames: no group of 10 fits 256 rows
    vx, vy = _grid(2, 10, -1.0, 1.0)
    with pytest.raises(mf.MFError) as e:
        mf.prf_plan(vx, vy, 140, kernel=2, group=10, segments=1)
    assert e.value.status == 5
    # shorter time segments bring the spread under the limit
    assert mf.prf_plan(vx, vy, 140, kernel=2, group=10)["window_rows"] <= 256
    info = mf.prf_plan(vx, vy, 140)  # the planner splits the columns instead
    assert info["kernel"] == 2 and info["window_rows"] <= 256


def test_segments_shrink_the_window(mf):
    """Within a time segment a CTA follows each trajectory from its position
    at the segment's first frame, so the window rows shrink roughly as the
    segment length; the planner splits the paper grid's frames."""
    vx, vy = _grid(10, 10)
    rows = {S: mf.prf_plan(vx, vy, 1000, kernel=2, group=5, tile_h=96, tile_w=32, segments=S)["window_rows"]
            for S in (1, 2, 4, 8)}
    assert rows[1] > rows[2] > rows[4] > rows[8] >= 96 + 4
    assert rows[1] - 100 > 3 * (rows[4] - 100)
    assert mf.prf_plan(vx, vy, 1000)["time_segments"] > 1
    # segments start on whole record chunks of 8 frames: 24 frames hold 3
    assert mf.prf_plan(vx, vy, 24, kernel=2, segments=3)["time_segments"] == 3
    with pytest.raises(mf.MFError):
        mf.prf_plan(vx, vy, 24, kernel=2, segments=4)


def test_shift_stack_plans_single_tap_passes(mf):
    # PRF kind 2 (one tap of 1 in the base pixel): the factored numerator
    # runs its single-tap passes; the Gaussian runs five taps
    vx, vy = _grid(10, 10)
    info = mf.prf_plan(vx, vy, 400, kind=2)
    assert info["kernel"] == 2 and info["taps"] == 1
    assert mf.prf_plan(vx, vy, 400)["taps"] == 5
    assert mf.prf_plan(vx, vy, 400, kind=1)["taps"] == 5
    with pytest.raises(mf.MFError):
        mf.prf_plan(vx, vy, 400, kind=3)


def test_measured_workloads_keep_their_plans(mf):
    # the layouts behind the measured numbers (1000 frames, |v| <= 0.1
    # px/frame): a change of the cost model that moves them must be measured
    vx, vy = _grid(10, 10)
    info = mf.prf_plan(vx, vy, 1000)
    got = {k: info[k] for k in ("kernel", "groups", "warps_per_group", "tile_h", "tile_w", "window_rows",
                                "stages", "time_segments", "taps")}
    assert got == {"kernel": 2, "groups": 10, "warps_per_group": 10, "tile_h": 64, "tile_w": 32,
                   "window_rows": 136, "stages": 5, "time_segments": 3, "taps": 5}
    vx, vy = _grid(40, 25)
    info = mf.prf_plan(vx, vy, 1000)
    assert (info["groups"], info["warps_per_group"], info["tile_h"], info["time_segments"]) == (120, 9, 64, 2)


def test_plan_with_frame_model(mf):
    # a frame model moves the base pixels, so the window rows and segments
    # follow it; the identity model is the linear plan
    vx, vy = _grid(10, 10)
    T = 400
    base = mf.prf_plan(vx, vy, T)
    same = mf.prf_plan(vx, vy, T, times=np.arange(T, dtype=float), jitter=np.zeros((T, 2)))
    assert same == base
    g = np.random.default_rng(3)
    jit = g.uniform(-1.5, 1.5, size=(T, 2))
    tau = np.arange(T, dtype=float) + np.where(np.arange(T) >= T // 2, 300.0, 0.0)
    info = mf.prf_plan(vx, vy, T, times=tau, jitter=jit)
    assert info["kernel"] == 2 and info["taps"] == 5
    assert info["max_abs_shift"] > base["max_abs_shift"]  # 700 cadences of motion instead of 400
    with pytest.raises(mf.MFError):
        mf.prf_plan(vx, vy, T, jitter=np.full((T, 2), np.nan))
    with pytest.raises(ValueError):
        mf.prf_plan(vx, vy, T, times=np.zeros(T + 1))


def test_factored_plans_stay_within_the_kernel_limits(mf):
    # every factored layout the planner picks fits the kernel it runs on:
    # at most 20 warps (the 640-thread launch bound), the shared-memory
    # budget of one CTA and a window of at most 256 rows, over grids of
    # different shapes, speeds and lengths
    rng = np.random.default_rng(11)
    for _ in range(40):
        nx, ny = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        vmax = float(rng.choice([0.02, 0.1, 0.3, 1.0]))
        T = int(rng.integers(8, 1300))
        vx, vy = _grid(nx, ny, -vmax, vmax)
        try:
            info = mf.prf_plan(vx, vy, T)
        except mf.MFError:
            continue
        if info["kernel"] != 2:
            continue
        warps = info["warps_per_group"] * (info["tile_h"] // 32) * (info["tile_w"] // 32)
        assert warps <= 20, (nx, ny, vmax, T, info)
        assert info["smem_bytes"] <= 227 * 1024 and info["window_rows"] <= 256, (nx, ny, vmax, T, info)
