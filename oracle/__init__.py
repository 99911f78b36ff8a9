"""CPU oracle for private ring linear algebra over additive secret shares.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the protocol definitions of CrypTen (arXiv 2109.00984, §5 and
Appendix D) in numpy uint64 arithmetic, whose wraparound is exactly the ring
Z/2^64.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The CUDA product path never imports, links
or executes anything here, and nothing here imports the CUDA package.

Modules
-------
prg         Philox4x64-10 counter PRG and the protocol's randomness streams.
fixed       Fixed-point encode / decode (§5.1).
sharing     Pseudorandom zero-share sharing and reveal (§5.1).
ring        Ring matmul and direct sliding-window convolution over Z/2^64.
dealer      Trusted-third-party material: Beaver triples, binary AND triples,
            random-bit pairs for B2A (§4 TTP, Appendix D.1.1-D.1.3).
beaver      Beaver multiplication for elementwise / matmul / conv (App. D.1.1).
truncation  Two-party local truncation (App. D.1.1).
binary      Binary AND, Kogge-Stone carry-lookahead adder, A2B, B2A (Alg. 2),
            comparator, private ReLU (§5.2, App. D.1.2-D.1.4).
transcript  Records every opening (round, bytes) for round-count checks.
nets        Compositions: the speech-shaped conv stack and its plaintext twin.

Parity status: every function here is pinned by a ``-m "not gpu"`` test that
does not re-run the function's own formula (see tests/test_oracle_*.py).
"""
