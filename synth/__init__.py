"""Seeded synthetic (protein, genomic region) pairs shaped like the paper's
workloads.  This module builds inputs only: it holds no alignment
arithmetic, and both the oracle tests and the GPU path consume what it
produces."""
from .gen import (Pair, config1, config2, config3, serving_pairs, random_protein,
                  reverse_translate, random_dna, revcomp, AA20, pairs_cells)
from .genome import GenomeWorkload, config5, regions_from_chains

__all__ = ["Pair", "config1", "config2", "config3", "serving_pairs", "random_protein",
           "reverse_translate", "random_dna", "revcomp", "AA20", "pairs_cells", "GenomeWorkload", "config5", "regions_from_chains"]
