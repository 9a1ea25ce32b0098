"""Host-side serving logic that needs no GPU: the admission footprint."""
import pytest


@pytest.fixture(scope="module")
def hz():
    from paper_2409_16172_gb300 import build
    build.build()
    from paper_2409_16172_gb300 import hz as _hz
    return _hz


def test_footprint_grows_with_every_dimension(hz):
    base = hz.request_footprint((256, 256), 6, 2, 1, 30, 1)
    assert hz.request_footprint((512, 512), 6, 2, 1, 30, 1) > 3.5 * base
    assert hz.request_footprint((256, 256), 12, 4, 1, 30, 1) > base
    assert hz.request_footprint((256, 256), 6, 2, 1, 40, 1) > base
    assert hz.request_footprint((256, 256), 6, 2, 1, 30, 4) > 3.5 * base
    # the FP64 path keeps no Z basis (one c128 work vector instead)
    assert hz.request_footprint((256, 256), 6, 2, 0, 30, 1) < base
    assert hz.request_footprint((64, 64, 64), 6, 2, 1, 30, 1) == hz.request_footprint(
        (64, 64, 64), 6, 2, 1, 30, 1)


def test_footprint_of_the_config2_workload(hz):
    # 1024^2, K = 16, FGMRES(40): basis 41 x 16 MiB, Z 40 x 8 MiB, planes 16 x 8 MiB
    fp = hz.request_footprint((1024, 1024), 12, 4, 1, 40, 1)
    n = 1024 * 1024
    assert fp >= n * (41 * 16 + 40 * 8 + 16 * 8)
    assert fp <= 1.5 * n * (41 * 16 + 40 * 8 + 16 * 8) + (64 << 20)


def test_footprint_counts_bivariate_planes_and_records(hz):
    """Bivariate (c, a) media hold (M + Mt) Ma planes per right-hand side and
    a 52-byte (node, weight) record per point; the quadratic basis only the
    record."""
    n = 512 * 512
    base = hz.request_footprint((512, 512), 12, 4, 1, 40, 1, has_a=True)
    biv = hz.request_footprint((512, 512), 12, 4, 1, 40, 1, has_a=True, Ma=3)
    assert biv - base >= n * (2 * 16 * 8 + 52)
    quad = hz.request_footprint((512, 512), 11, 4, 1, 40, 1, has_a=True, basis=1)
    lin = hz.request_footprint((512, 512), 11, 4, 1, 40, 1, has_a=True)
    assert quad - lin >= n * 52
    assert hz.request_footprint((512, 512), 12, 4, 1, 40, 1, has_a=True, Ma=1) == base
