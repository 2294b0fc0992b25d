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
    # depth-sorted lists add the sort + split; deterministic mode also places
    # the pair slots and gathers them
    assert bench.kernels_per_step("alpha", (16, 8)) == per_frame + it * 9
    assert bench.kernels_per_step("oit", (16, 8), deterministic=True) == per_frame + it * 11
    # the per-Gaussian schedule: pixel terms + per-Gaussian backward, no sort
    assert bench.kernels_per_step("oit", (16, 8), schedule="per-gaussian") == per_frame + it * 9
