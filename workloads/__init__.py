"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path."""
from .problems import *  # noqa: F401,F403
