"""FP64 CPU oracle for PISCO's pixel-space convolution (arXiv:1908.05662).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The CUDA library never links, imports or calls it,
and this package shares no code with the CUDA path.

The oracle is a plain, slow, obviously-correct restatement of the paper:

* ``healpix``   -- HEALPix RING pixel centres and the disc query (Sec. 5.1 and
                   Sec. 5.2: "sky pixels inside the beamsor extension").
* ``geometry``  -- sky and antenna bases (Sec. 2), the antenna coordinates
                   (rho, sigma) and the co-polarisation angle chi, both by the
                   spherical-trigonometry route of Appendix A and by the vector
                   route of Sec. 2 (Ludwig's third definition).
* ``beam``      -- the tangent-plane beam grid, its bilinear re-pixelisation
                   (Sec. 4.2) and the normalisation Omega~ (Sec. 3).
* ``convolve``  -- the pixelised convolution d(q0) of Sec. 4.2
                   (eq. discrete_beam_conv_tensor), its transpose with respect
                   to the sky (TOD -> I,Q,U maps) and with respect to the six
                   beam grids.

Everything is float64.  Every function cites the passage it follows.
"""

from . import healpix, geometry, beam, convolve  # noqa: F401
