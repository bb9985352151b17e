"""FP64 CPU oracle for the line-by-line opacity cross-section path.

TEST INFRASTRUCTURE ONLY. This package is imported, called or executed only by
`tests/`, `__graft_entry__.smoke()` and the CPU-baseline / reference leg of
`bench.py`. The product path (the CUDA library and its Python binding) never
imports it and shares no code, table or constant with it.

It is a plain, slow, obviously correct FP64 restatement of what the pyROX paper
computes ("Functionality of pyROX": line strengths and broadening widths at each
(P,T); Voigt profiles as the real part of the Faddeeva function evaluated with
scipy.special.wofz; profiles summed into a cross-section for each
temperature-pressure point). The paper prints no formula; the standard HITRAN /
ExoMol definitions it relies on are stated in `rox_oracle.py`, each with the
reading taken where the paper is silent.
"""
from .rox_oracle import *  # noqa: F401,F403
