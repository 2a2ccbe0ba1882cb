"""Plain CPU oracle of the SH block-texture codec (test infrastructure only)."""
