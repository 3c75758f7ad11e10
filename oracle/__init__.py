"""CPU oracle for the batched trajectory optimizer -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct FP64 implementation of what the CUDA path
computes, written from the thesis (Algorithm 2 of Paper II, the projection
optimizer and sampler of Paper III, and the warm-start network that the
thesis leaves as future work). Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. It shares no code with
the CUDA library and neither side imports the other; both consume the seeded
inputs of ``paper_2408_10731_b300.scenes``.

Parity status per function is stated in each module's header.
"""
