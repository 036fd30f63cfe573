"""Plain FP64 CPU oracle for the hybrid IB/phase-field step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and
``--impl reference``) may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs it.
"""
