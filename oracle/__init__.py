"""FP64 CPU oracle for HoloGen's phase-retrieval hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  It shares no code with the CUDA library (no tables, no
helpers, no headers) and never imports it.

The paper (section "Algorithm Libraries") names the pieces -- Gerchberg-Saxton and other iterative
Fourier transform algorithms (HoloGenAlgGSCuda), One-Step Phase-Retrieval (HoloGenAlgOSPRCuda),
Fourier and Fresnel holograms (keywords), an FFT handler (FFTHandlerCuda), a quantiser
(QuantiserCuda), a normaliser and a randomiser -- but prints no equation for any of them.  Each
module therefore writes out the published method the name refers to (Gerchberg & Saxton 1972;
Fienup 1982; Cable, Buckley et al. 2004; Pasienski & DeMarco 2008; Seldowitz, Allebach & Sweeney 1987; Goodman's single-FFT Fresnel
transform; Kingma & Ba 2015; Salmon et al. 2011) in plain numpy float64, and every reading taken where the paper is silent is
stated in the docstring of the function that takes it.

Pins (see tests/test_oracle_*.py): closed forms (delta, plane wave, Gaussian chirp transform),
brute-force DFT sums, Parseval, inverse-of-forward, the error-reduction property of GS, the GS fixed
point, brute-force nearest-level quantisation, Philox known-answer vectors, finite differences of
the gradient-descent loss.  Parity with the paper itself is unpinned: the paper prints no values.

Modules:
  dft       naive O(N^2) DFT and brute-force 2D sums (unitary convention)
  fft       own mixed-radix Stockham FFT (any length; radices 4, 2, 3, 5, other primes)
  optics    single-FFT Fresnel chirp and propagation
  project   SLM-plane projections (continuous / N-level / binary) and amplitude replacement
  metrics   optimal-scale intensity NMSE
  gs        Gerchberg-Saxton (single plane) and averaged-projection multi-plane GS
  mraf      mixed-region amplitude freedom (signal window, mixing m), hybrid input-output, and
            region-of-interest NMSE
  dbs       direct binary search with the single-pixel replay update
  philox    Philox4x32-10 counter-based generator
  ospr      One-Step Phase-Retrieval
  gd        gradient-descent (Wirtinger) loss, analytic gradient and Adam
"""
from . import dft, fft, optics, project, metrics, gs, philox, ospr, gd  # noqa: F401
