"""CPU oracle for the relational hot path (filter -> hash join -> group-by aggregation).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference arm of ``bench.py`` may import or call anything in this package.
The product path (the CUDA library and its Python binding) never touches it and shares no code
with it.
"""
from .relational import *  # noqa: F401,F403
from .relational import __all__ as _rel_all
from .strings import *  # noqa: F401,F403
from .strings import __all__ as _str_all
from .chunked import *  # noqa: F401,F403
from .chunked import __all__ as _chunk_all

__all__ = list(_rel_all) + list(_str_all) + list(_chunk_all)
