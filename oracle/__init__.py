"""FP64 CPU oracle for the simulation and pre-processing hot path (test infrastructure).

This package is the slow, plain, obviously-correct restatement of what the GPU
library computes.  It exists only to check the GPU path: the only code allowed
to import it is ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference legs of ``bench.py``.  The product path (the ``paper_2407_19048_gb300`` package and
its CUDA library) never imports, calls or links anything here, and this package
imports nothing from the product.

The method (Sec. 3, simulation on accelerated hardware) generates training
data on the fly: draw parameters from the prior (Table 1), evaluate
frequency-domain compact-binary waveforms (Sec. 3.1), project them onto the
detectors, inject them into background strain, estimate the background power
spectrum and whiten the batch (Sec. 3.2).  The plain likelihood used by the
paper's nested-sampling comparison (Sec. 6, Fig. 5 caption: the usual
Gaussian-noise GW likelihood) is the sixth piece, and importance weights built on it the seventh.

Modules, in pipeline order:

* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al. 2011).
* ``prior``      -- parameter draws for one batch (Table 1 / configured ranges).
* ``taylorf2``   -- TaylorF2 3.5PN frequency-domain inspiral (Sec. 3.1).
* ``detector``   -- detector geometry, antenna patterns, delays, projection.
* ``noise``      -- analytic aLIGO PSD and coloured Gaussian background.
* ``spectral``   -- Welch PSD, PSD interpolation, injection, whitening.
* ``likelihood`` -- noise-weighted inner product, log-likelihood, mismatch.
* ``importance`` -- importance weights, effective sample size, evidence per event.
* ``gemm``       -- bfloat16 dense products and the dense layer, forward and backward.
* ``learn``      -- the learned Gaussian proposal: features, loss, AdamW, proposal density.
* ``flow``       -- the conditional coupling flow: embedding, coupling layers, loss and its
  gradient, base draws, the proposal map to theta and the prior-to-proposal ratio.
* ``resnet``     -- the ResNet-1D data summary of Sec. 4, forward and backward.
* ``vicreg``     -- VICReg pre-training of the summary (Sec. 4.1): loss, gradient, view re-timing.
* ``skymap``     -- HEALPix pixels, sky maps from weighted draws and per-pixel flow densities (Sec. 5).
* ``iaf``        -- the paper's inverse-autoregressive flow (Sec. 5.1): MADE masks,
  sampling, the D-pass density and the training gradient (a variant the library's
  kernels do not build yet).
* ``pipeline``   -- the whole per-batch pass, step by step, unfused.

Everything is float64 / uint32-uint64 numpy.  ``numpy.fft`` is used as the
FFT primitive; the pins in ``tests/test_oracle_*.py`` tie every function to
closed forms, textbook special cases, library routines (``scipy.signal``) or
brute force.

Parity status: every function is pinned except the spin-dependent TaylorF2
terms beyond 1.5PN spin-orbit, which the oracle does not include (no
published table for them is available here), and IMRPhenomD, which is not
implemented (its fitted coefficient tables are not available).
"""
