"""CPU FP64 oracle for the Haar-domain non-linear phase shift and the
per-vertex double product (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1705_07272_gb300``): it is a plain, slow restatement of what the
paper's run-time path computes, written for checking by eye:

* ``haar``       - orthonormal 2-D non-standard Haar transform of a lat-long
                   map and its canonical coefficient order;
* ``resample``   - the lat-long map's extension across the poles and the
                   azimuth seam, bilinear sampling, the translation and the
                   rotation g(theta, phi) = f(Theta, Phi) of Eq. (theta)/(phi);
* ``shift``      - the phase shift itself: Haar(resample(Haar^-1 c));
* ``transport``  - projection of transport weights to Haar, top-K / lowest-K
                   truncation, CSR packing, BF16/FP16 storage rounding;
* ``shade``      - the double product, by brute force in pixel space;
* ``paper_route``- the paper's own derivative route (difference fields,
                   triangle and box kernels, a-trous recursion) used as an
                   independent pin of the exact operator;
* ``mlp``        - FP64 forward/backward of the transport surrogate.
"""
