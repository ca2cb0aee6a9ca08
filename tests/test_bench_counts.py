"""The benchmark's roofline numerators and accuracy measure (host logic, no
GPU): the algorithmic flops and bytes of one objective + gradient
evaluation follow the counts of the data term (Eq. 2-8: per voxel and scan
16 transverse, 8 axial and 20 adjoint-gradient multiply-adds, about 8 flops
of loss per voxel pair; both volumes read once, the en-face images, the
float64 displacement, the float gradient and the two per-A-scan partials),
and the RMS against the synthetic truth keeps only the masked A-scans
inside the border."""
import numpy as np

import bench


def test_flops_per_evaluation_clinical_size():
    # 300 x 300 A-scans x 512: 184 flop per voxel pair
    assert bench.flops_per_eval(300, 300, 512) == 300 * 300 * 512 * (2 * (16 + 8 + 20) * 2 + 8)
    assert bench.flops_per_eval(300, 300, 512) == 8.47872e9


def test_bytes_per_evaluation_by_storage():
    # float32: 2 * 512 * 4 volume bytes + 8 angio + 48 displacement + 32 outputs per A-scan
    assert bench.bytes_per_eval(300, 300, 512) == 300 * 300 * (2 * 512 * 4 + 8 + 48 + 32)
    assert bench.bytes_per_eval(300, 300, 512) == 376.56e6
    # 16-bit storage halves the volume bytes only
    assert bench.bytes_per_eval(300, 300, 512, s=2) == 300 * 300 * (2 * 512 * 2 + 88)


def test_rms_against_truth_uses_masked_ascans_inside_the_border():
    rng = np.random.default_rng(0)
    h, w = 20, 24
    T = rng.normal(size=(2, 3, h, w))
    mask = np.ones((2, h, w), dtype=bool)
    mask[0, 10, 12] = False
    D = T.copy()
    D[:, :, :4, :] += 100.0          # inside the 4-px border: ignored
    D[0, :, 10, 12] += 100.0         # masked out in scan X: ignored there
    D[1, :, 10, 12] += 1.0           # kept in scan Y
    a, r = bench.rms_vs_truth(D, T, mask)
    kept = (2 * (h - 8) * (w - 8) - 1) * 3
    assert a == np.sqrt(3 * 1.0 / kept)
    # the relative mode (X - Y) is taken only where both scans are valid
    assert r == 0.0
