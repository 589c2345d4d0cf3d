"""Algorithmic FLOP counts of the chain code (see count.py)."""
