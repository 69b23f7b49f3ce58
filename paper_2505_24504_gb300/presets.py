"""Solver configurations of the measured workloads.

The preconditioner schedule (the mg key of Sec. 4 and the pseudo-time factors
sigma of Sec. 3.5) and the launch shapes below were picked on a GB300 by timing
implicit steps per candidate (`autotune.tuned_schedule_context` searches the
same candidates: keys, then sigma_fv, then sigma_dg) and the kernels per launch
shape (`jfnk_autotune`).  They are recorded here so that the benchmark, the parity tests
at full size and the CPU reference all run the same configuration;
`bench.py --tune` runs the autotuner again and reports what it picks.  None of
these choices changes the converged answer (the Newton tolerance decides it);
they change iteration counts and speed only.
"""

# Warm bubble, DG Q3 on 160 x 80 quads, 5 FV levels, SDIRK2 at 20x the acoustic
# CFL step, FP32 preconditioner.
WARM_BUBBLE_Q3_160x80 = dict(mg_key="mg131211V", sigma_fv=1.0, sigma_dg=0.9,
                             tile_faces=64, tile_volume=1, tile_fv=128, fv_split_cells=4096)


def schedule(preset: dict) -> dict:
    """The schedule part of a preset (what the FP64 oracle also takes)."""
    return {k: preset[k] for k in ("mg_key", "sigma_fv", "sigma_dg")}
