"""FP64 CPU oracle of the hybrid chemotaxis step (test infrastructure only;
the GPU package never imports it)."""
