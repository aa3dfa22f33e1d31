"""FP64 CPU oracle for the Laplace kiFMM (test infrastructure, not part of the product).

Plain, slow, obviously correct restatements of what the GPU path computes:
  * `direct`  - the field sum of Eq. 1 with the Laplace kernel of Eq. 2 (NumPy and plain C);
  * `tree`    - domain, Morton keys, stable sort, leaves, levels, U and V lists (Section 2.1,
                Table 1), with brute-force list constructions straight from the definitions;
  * `kifmm`   - Algorithm 1 (uniform branches) with per-level operators built from actual box
                geometry, uncompressed M2L, and its transpose (the adjoint pass);
  * `adaptive` - the adaptive tree, its U, V, W and X lists, and Algorithm 1 with XLI and WLI;
  * `partition`, `distributed`, `samplesort` - Section 3's setup (with the sample sort of its
                step 1) and runtime over ranks;
  * `fft_m2l` - the M2L as a lattice convolution evaluated by FFT.

It shares no code with the CUDA library and never imports it.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may use it.  Inputs come from the `synth` module.
"""
