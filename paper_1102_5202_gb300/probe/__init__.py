"""Measurement probes: ``python -m paper_1102_5202_gb300.probe`` builds and runs the FP64/FP32
FMA-throughput probe (``alu_peak.cu``) on the current GPU."""
