"""Seeded synthetic inputs shared by tests and the benchmark (no solver arithmetic)."""
