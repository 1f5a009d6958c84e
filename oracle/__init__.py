"""FP64 CPU oracle of the receiver chain.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run anything in this
package.  It shares no code with the CUDA library and does not import it;
its only shared dependency is the seeded input generator
``paper_2108_07004_gb300.synth``, which holds none of the receiver's
arithmetic.

Every function follows the plain definition of its step (numpy FFTs are the
only library primitive used as a step).  Where the paper (arXiv 2108.07004)
is silent, the reading taken is stated in the docstring.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, an invariant, a physics
fact or brute force, except ``gs4d64`` table design (the authors' own
constellation is not printed: parity with it is unpinned).  ``mlp`` is the
learned demapper (forward, BCE, backward, Adam), pinned by identities,
finite differences and closed forms.  ``kk`` is the Kramers-Kronig
front-end (intensity -> field by the frequency-domain Hilbert transform),
pinned by the library's analytic-signal routine, exact minimum-phase tones
and the KK reconstruction error against CSPR.  ``fde`` is the trained static
frequency-domain equaliser with 4-to-2 resampling, pinned by the library
least-squares solve, exact inversion of a short pulse, exact resampling of
frame-periodic tones and the EVM gain after the KK front-end.
"""
from .formats import OracleFormat, oracle_format  # noqa: F401
from . import chain  # noqa: F401
from . import mlp  # noqa: F401
from . import kk  # noqa: F401
from . import fde  # noqa: F401
