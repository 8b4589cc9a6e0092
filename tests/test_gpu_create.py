"""Creation of large lattices: the upload of the fields in chunks of planes
overlapped with the pack of the chunks already there.

A lattice of at least 2^22 sites without per-link factors uploads F, omega
and the mask chunk by chunk and packs each chunk (Eq. 1 weights, Eq. 7
rotation) as soon as its upper neighbour plane has arrived; a lattice with
per-link factors takes the whole-array path.  With alpha = 1 and every link
factor 1 both give the same weights, so the two paths are compared bit for
bit on the weights, the rotation and the mask, with periodic and walled z,
reservoir faces, FP32 and BF16 weights; the stepped state agrees too.
"""
import numpy as np
import pytest

import lpc_inputs

pytestmark = pytest.mark.gpu

RES = ((-0.75, 1.25, 0.5 - 0.25j), (0.5, 0.625, 1.0 + 0.0j), (0.25, 0.75, 0.0j), (-1.5, 2.0, 0.0j),
       (-0.25, 1.5, 0.75 + 0.5j), (0.75, 0.5, 0.25 - 0.5j))

# (nz, ny, nx), periodic (x, y, z), reservoir faces, weight type
CASES = [
    ((40, 128, 1024), (1, 1, 1), (), 0),        # 5.2e6 sites, eight chunks of 5 planes, z wraps
    ((37, 96, 1200), (1, 1, 0), (), 1),         # ragged chunks, z walls, BF16
    ((11, 300, 1300), (0, 1, 1), (0, 1), 0),    # fewer planes per chunk than 2, x reservoirs
    ((20, 160, 1400), (1, 1, 0), (4, 5), 0),    # z reservoirs: the lattice holds a halo plane on each side
]


@pytest.mark.parametrize("shape,periodic,faces,wdt", CASES)
def test_chunked_upload_and_pack_equal_the_whole_array_path(shape, periodic, faces, wdt):
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case(shape, 380 + shape[0], periodic=periodic, solid_frac=0.3, F_sd=1.5,
                                 shift_sd=5.0, alpha=1.0, msd_axes=0, weight_dtype=wdt)
    assert inp.n_sites >= 1 << 22
    kw = dict(reservoirs=tuple(RES[f] if f in faces else None for f in range(6))) if faces else {}
    chunked = Lattice.from_input(inp, **kw)
    whole = Lattice.from_input(inp, alpha_links=np.ones((3,) + tuple(shape)), **kw)
    try:
        assert np.array_equal(chunked.solid_mask(), inp.solid)
        assert np.array_equal(chunked.solid_mask(), whole.solid_mask())
        wc, ww = chunked.weights(), whole.weights()
        assert np.array_equal(wc, ww)
        assert np.count_nonzero(wc) > 0
        assert np.array_equal(chunked.rotation(), whole.rotation())
        chunked.step(5)
        whole.step(5)
        assert np.array_equal(chunked.density(), whole.density())
        assert np.array_equal(chunked.magnetization(), whole.magnetization())
    finally:
        chunked.close()
        whole.close()
