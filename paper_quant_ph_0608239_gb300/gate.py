"""The gate record of the Python binding.

A gate names its kind (``H X Y XB YB NOT R V SU2 U SWAP``, the kinds of
``qsim_gate.kind`` in ``include/qsim.h``), its target qubit(s), its control
qubits and its kind-specific parameters.  The binding marshals any object with
these four fields, so gate lists from other sources need no conversion.
"""
from collections import namedtuple

Gate = namedtuple("Gate", ["kind", "targets", "controls", "params"])
