"""Peak-throughput probe (measurement only): python -m paper_1510_08642_gb300.probes"""
