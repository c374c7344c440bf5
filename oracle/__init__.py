"""Oracle for the in-place truncated Fourier transform (Harvey & Roche, 2010).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct CPU
statement of what the GPU library computes.  Only ``tests/``, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import or
call it.  The CUDA library never routes through it, shares no code, header,
table or constant generator with it, and it imports nothing from the library.

Contents
--------
``oracle.field``   the three rings Z/p and the compatible roots of unity
                   omega_[k] (Section 2.2) fixed by one generator per prime.
``oracle.tft``     the definition (Section 2.2: F^_s = F(omega_s)), a brute
                   force inverse, Algorithm 1 (InplaceTFT) and Algorithm 2
                   (InplaceITFT) walked literally over the implicit tree of
                   Section 3, a textbook radix-2 FFT, schoolbook products, the
                   TFT product (Section 5, first paragraph) and Algorithm 3.
``oracle.native``  ctypes wrapper around ``oracle/alg_c.c``: the same
                   Algorithm 1 / Algorithm 2 / definition in plain C with
                   ``unsigned __int128 % p`` arithmetic, for sizes the Python
                   loops cannot reach in seconds.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
properties the paper or elementary algebra fixes (brute-force evaluation,
Gaussian elimination, the textbook FFT at n = 2^k, truncation of the padded
transform, schoolbook products, Figure 1's tree, visit counts).  The paper
prints no numeric worked example, so individual transform *values* are pinned
through the definition and the root convention only.
"""
