"""FP64 CPU oracle of the staggered-mesh EB advance (test infrastructure only)."""
