"""The seeded generators: reproducible, with the stated structure."""
import numpy as np

from paper_1009_0958_gb300 import synth


def test_deterministic():
    a = synth.make_image(50, 70, 3, 0.1, rectangles=12)
    b = synth.make_image(50, 70, 3, 0.1, rectangles=12)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    c = synth.make_image(50, 70, 4, 0.1, rectangles=12)
    assert not np.array_equal(a[1], c[1])


def test_field_range_and_noise_fraction():
    clean = synth.sinusoid_field(256, 256, 0)
    assert clean.dtype == np.uint8 and clean.shape == (256, 256, 3)
    assert clean.min() > 0                          # no black pixel in the field
    for phi in (0.05, 0.1, 0.2):
        noisy = synth.impulsive_noise(clean, phi, 1)
        frac = np.any(noisy != clean, axis=2).mean()
        assert abs(frac - phi) < 0.01               # an impulse may equal the original


def test_channel_model_eq8():
    clean = synth.sinusoid_field(200, 200, 2)
    noisy = synth.impulsive_noise(clean, 0.5, 3, channel_probs=(0.25, 0.25, 0.25))
    changed = (noisy != clean).sum(axis=2)
    single = (changed == 1).sum() / (changed > 0).sum()
    assert 0.6 < single < 0.85                      # 3 x 0.25 single-channel, 0.25 all-channel


def test_float_conversion_and_batch_shapes():
    _, img = synth.make_image(8, 9, 0)
    f = synth.to_float_nchw(img)
    assert f.shape == (1, 3, 8, 9) and f.dtype == np.float32 and f.max() <= 1.0
    shapes = synth.batch_shapes(256, 0)
    assert len(shapes) == 256 and min(min(s) for s in shapes) >= 1
    sides = np.sqrt([m * n for m, n in shapes])
    assert 40 <= sides.min() and sides.max() <= 2100
