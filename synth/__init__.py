"""Seeded synthetic inputs (graphs, sources, signals) shared by the oracle tests and the CUDA path."""
