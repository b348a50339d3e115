"""B300-native phasor-PIC hot path (arXiv 2609.15043): an RZ PIC/MCC step for
an argon ICP with per-RF-period phasor coupling to a turn-resolved coil
circuit, behind the C-ABI library ``libphasorpic.so``.

``phasorpic`` is the ctypes binding (argument marshalling only); ``workloads``
holds the seeded synthetic inputs.
"""
