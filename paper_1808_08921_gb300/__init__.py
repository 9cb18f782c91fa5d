"""GB300 (sm_103a) coupled lattice-Boltzmann / DEM time step of
"Hydro-micromechanical modeling of wave propagation in saturated granular
media" (arXiv 1808.08921), behind the C ABI declared in include/lbmdem.h.

    from paper_1808_08921_gb300 import lbmdem
    sim = lbmdem.Sim.from_workload(workload)
    sim.step(100)
    rho, u, solid = sim.fields()
"""
__all__ = ["lbmdem", "build"]
