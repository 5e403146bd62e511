"""CPU FP64 oracle of the contrail finite-volume step -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this
package.  It shares no code with the CUDA library in paper_2504_20742_gb300/ and neither
imports the other.
"""
from .oracle import (  # noqa: F401
    build,
    Oracle,
    ln_psat_l,
    ln_psat_i,
    tsat,
    sigma_lg,
    growth,
    koop_log10J,
    hfg,
    roe_flux,
    roe_c2,
    dv_mol,
    table_eval,
    diffusive_flux,
    source_batch,
    prim_to_cons_batch,
    cons_to_prim_batch,
    const,
    NF,
    NDIAG,
    AUX_NAMES,
)
