"""CPU oracle for the sparse-sampling-and-completion VPL renderer (TEST INFRASTRUCTURE).

This package is a plain, slow, float64 restatement of what the paper computes.  It
exists only to check the CUDA library: only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path (no kernels, headers, tables or helpers) and never imports it; both sides
read the same seeded inputs from ``ltinputs``.

Modules and the passages they follow (Huo et al., "Sparse Sampling and Completion
for Light Transport in VPL-based Rendering"):

  philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11), the
              source of every random choice of the method
  shading     entry A(i,j) of the lighting matrix (Sec. 3, problem statement) and
              the shadow-ray visibility test (Sec. 6, ray casting)
  bruteforce  the image as the column sum of the full lighting matrix (Sec. 3)
  tree        light tree over the VPLs (Sec. 3 step 1; Sec. 4 I_f = I_a + I_b)
  cut         conservative global light cut (Sec. 3 step 1, Sec. 6)
  slices      matrix slicing by clustering position+normal (Sec. 3 step 2)
  pass1       first sampling pass and light coarsening (Sec. 4, Eq. 2)
  pass2       second sampling pass from pdf(i,j) ~ f(i) g(j) (Sec. 5, Eq. 3)
  als         masked alternating least squares completion (Sec. 5; the paper's
              factor form M = X Y, rank q)
  render      the image from the factors, X (Y e) (Sec. 3 step 5)
  pipeline    the five steps end to end
  proposal    the learned pass-2 proposal (an extension the paper leaves to future
              work): features, leverage targets, the bfloat16 MLP, its gradients
              and Adam

Every readings of a passage that the paper leaves open is stated in the docstring
of the function that takes it.
"""
