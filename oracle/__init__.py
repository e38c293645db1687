"""Plain CPU oracle of the TPC sector tracker (test infrastructure only)."""
