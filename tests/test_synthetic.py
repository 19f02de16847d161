"""The seeded input generators (CPU): the tiled evaluation used for paper-size slices gives the
stack of the dense evaluation."""
import torch

from paper_1506_02079_gb300.synthetic import evaluate_stack, evaluate_stack_tiled, stack_params


def test_tiled_generator_equals_dense_generator():
    """Tiles that split blob footprints (64 and 100 do not divide 300 x 517), and a z sub-range,
    give the dense evaluation's values in FP64; in FP32 the uint8 stack differs by at most one
    grey level on a few voxels (rounding of values that sit near a half)."""
    p = stack_params(5, 300, 517, seed=4)
    dense = evaluate_stack(p, dtype=torch.float64, out_dtype=torch.float64)
    for tile in (64, 100):
        t = evaluate_stack_tiled(p, dtype=torch.float64, out_dtype=torch.float64, tile=tile)
        assert float((t - dense).abs().max()) <= 1e-9
    sub = evaluate_stack_tiled(p, z0=1, z1=4, dtype=torch.float64, out_dtype=torch.float64, tile=128)
    assert float((sub - dense[1:4]).abs().max()) <= 1e-9
    u8 = evaluate_stack_tiled(p, dtype=torch.float32, out_dtype=torch.uint8, tile=128)
    d8 = evaluate_stack(p, dtype=torch.float64, out_dtype=torch.uint8)
    diff = (u8.int() - d8.int()).abs()
    assert int(diff.max()) <= 1 and float((diff > 0).float().mean()) < 1e-4


def test_tiled_generator_writes_into_a_given_buffer():
    p = stack_params(3, 70, 90, seed=1)
    buf = torch.full((2, 70, 90), 7, dtype=torch.uint8)
    out = evaluate_stack_tiled(p, z0=1, z1=3, tile=32, out=buf)
    assert out is buf
    assert torch.equal(buf, evaluate_stack_tiled(p, z0=1, z1=3, tile=70))
