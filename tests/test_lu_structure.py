"""The nested-dissection analysis of the sparse LU (lrfsi_lu_info; host only,
no GPU): it succeeds on the benchmark meshes (every separator separates,
every matrix entry falls in its front), and it needs far less work and memory
than the slab-ordered block LU on the larger meshes, with fronts no wider than
one vertex line of the channel (2 ny + 1 nodes) or a leaf region of at most
5 x 5 nodes."""
import pytest

from paper_2008_10275_gb300 import build, lrfsi


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lrfsi.load()


@pytest.mark.parametrize("nx,ny", [(20, 4), (80, 16), (40, 8), (10, 2)])
def test_nested_dissection_analysis(nx, ny):
    info = lrfsi.lu_info(nx, ny)
    # a vertical separator: 2 ny + 1 nodes with 4 unknowns and ny + 1 pressures;
    # a leaf: at most 25 nodes with 4 unknowns and 9 pressures
    assert info["max_separator"] <= max(4 * (2 * ny + 1) + ny + 1, 4 * 25 + 9)
    assert info["fronts"] >= 3 and info["heights"] >= 2
    assert info["factor_flops"] > 0 and info["factor_doubles"] > 0
    if nx >= 80:
        assert info["factor_flops"] * 5 < info["slab_lu_flops"]
        assert info["factor_doubles"] < info["slab_lu_doubles"]


def test_large_mesh_fits_where_the_slab_lu_did_not():
    info = lrfsi.lu_info(320, 64)
    assert info["factor_doubles"] * 8 < 4e9          # < 4 GB per factorisation (slab LU: 12.4 GB)
    assert info["factor_flops"] * 20 < info["slab_lu_flops"]
    assert info["max_separator"] <= 800              # the panel kernel's limit
