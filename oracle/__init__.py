"""CPU oracle for the OVRO-LWA ultra-narrowband imaging hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
reference written from the paper (exact integers where the method is integer,
FP64 elsewhere).  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import it.  The CUDA library
(``paper_2606_04304_gb300``) never imports, links or calls anything here, and
nothing here imports the CUDA library: the two share only the seeded input
generator (``synth``), which holds none of the method's arithmetic.

Modules and the paper passages they follow:

* ``upchan``   Section 2.1: unpack the F-engine's coarse-channel voltages and
               upchannelize with an FFT over time samples; 8-bit requantisation
               for the correlator input (xGPU takes 8-bit complex samples).
* ``xengine``  Section 2.1: cross-correlate every antenna pair and polarisation
               product per fine channel, integrated over the spectra.
* ``imaging``  Section 2.2: dirty all-sky image per fine channel (uv gridding
               with a prolate-spheroidal kernel, 2D FFT, grid correction).
* ``detect``   Section 2.4: MAD standardisation, running-median high-pass,
               boxcar matched filters (1-100 channels), Benjamini-Hochberg FDR,
               1D non-maximum suppression along frequency.
* ``scorer``   the learned candidate scorer (not in the paper): a small MLP on
               (pixel, channel) cutouts, forward/backward/Adam in FP64.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, library routines or brute force on tiny inputs.
"""
