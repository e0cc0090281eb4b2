"""Peak microbenchmarks: the measured denominators of the ALU rooflines.

Built by :func:`paper_1612_06592_gb300.build` into ``_build/libmb.so``; run
with ``python -m paper_1612_06592_gb300.microbench.peaks`` on the GPU, which
writes ``profiles/fp32_peak.json``.  Not part of the pipeline.
"""
