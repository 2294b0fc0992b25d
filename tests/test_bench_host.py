"""Host logic of bench.py (CPU): the kernel launches it claims per step
(`gpu_launches`) for each form of the iteration, from the kernels each form
launches per iteration (plus fusion and ray-cast once per frame)."""
import bench


def test_kernels_per_step_counts_each_form():
    per_frame = 2  # fuse, ray-cast
    it = bench.ITERS_PER_FRAME
    # default: project, scan, emit, composite, finalize, carry-over backward,
    # projection adjoint + Adam, step counter
    assert bench.kernels_per_step("oit", (16, 8)) == per_frame + it * 8
    # the two-call backward + Adam adds the separate Adam kernel
    assert bench.kernels_per_step("oit", (16, 8), fused=False) == per_frame + it * 9
    # depth-sorted lists add the sort + split; deterministic mode with OIT
    # needs the block prefix for its fixed-order lists up to 6144 tiles (no
    # sort) and nothing more in the backward (the fused loss's bounds come
    # from the forward, a memset zeroes the fixed-point sums, the projection
    # adjoint converts them); with alpha it places and gathers pair slots
    assert bench.kernels_per_step("alpha", (16, 8)) == per_frame + it * 9
    assert bench.kernels_per_step("oit", (16, 8), deterministic=True) == per_frame + it * 9
    assert bench.kernels_per_step("oit", (8, 8), deterministic=True,
                                  size=(1280, 720)) == per_frame + it * 9
    assert bench.kernels_per_step("alpha", (16, 8), deterministic=True) == per_frame + it * 11
    # the per-Gaussian schedule: pixel terms + per-Gaussian backward, no sort
    assert bench.kernels_per_step("oit", (16, 8), schedule="per-gaussian") == per_frame + it * 9


def test_kernels_per_step_counts_the_split_of_large_tile_grids():
    """Unsorted lists are binned straight into tiles only while a view's tile
    grid fits the binning histogram (16384 tiles); beyond that they go
    through super-tiles and a split kernel."""
    per_frame = 2
    it = bench.ITERS_PER_FRAME
    # 1280x720 with 16x8 tiles: 80 x 90 = 7200 tiles, binned straight into tiles
    assert bench.kernels_per_step("oit", (16, 8), size=(1280, 720)) == per_frame + it * 8
    # 4096x2160 with 8x8 tiles: 512 x 270 = 138240 tiles: + the split
    assert bench.kernels_per_step("oit", (8, 8), size=(4096, 2160)) == per_frame + it * 9
    assert bench.kernels_per_step("oit", (8, 8), size=(4096, 2160),
                                  schedule="per-gaussian") == per_frame + it * 10
    # depth-sorted lists split anyway
    assert bench.kernels_per_step("alpha", (8, 8), size=(4096, 2160)) == per_frame + it * 9
