"""CPU baselines timed by bench.py (not the product, not the oracle)."""
