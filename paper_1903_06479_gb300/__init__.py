"""GB300-native npFEM red-blood-cell solver hot path (arXiv:1903.06479).

The compute path is the C-ABI library ``libnpfem.so`` built from ``csrc/``; the
Python side only marshals arguments (see ``npfem``)."""
