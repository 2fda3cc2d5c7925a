"""Seeded synthetic ACOPF grids and KKT systems (problem data shared by the
oracle and the GPU path; contains no linear-solver arithmetic)."""
from .grid import Grid, make_grid
from .kkt import KKTPattern, KKTPoint, WORKLOADS, branch_terms, line_terms, mu_schedule
from .opf import OPFData, flat_start, opf_data

__all__ = ["Grid", "make_grid", "KKTPattern", "KKTPoint", "WORKLOADS",
           "branch_terms", "line_terms", "mu_schedule", "OPFData", "flat_start", "opf_data"]
