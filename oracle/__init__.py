"""CPU oracle of the PERKS hot path.  Test infrastructure only (see oracle.py)."""
