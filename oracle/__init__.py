"""Plain FP64 CPU oracle of the phase-field lattice Boltzmann model (test infrastructure only)."""
