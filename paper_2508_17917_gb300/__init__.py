"""GB300 nodal interior-penalty DG solver for 2D compressible Navier-Stokes.

Python binding of the C-ABI library ``libdg.so`` (declared in include/dg.h).
Every entry point is the C function of the same name; this package only
marshals arguments.  Importing it loads the library and raises if it has not
been built: there is no CPU fallback.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401
