"""Seeded synthetic inputs for the counting-query workloads.

This package only draws random inputs (databases, query lists, itemsets,
transaction bitmaps).  It holds none of the counting or scoring arithmetic, so
the CUDA path and the CPU oracle can both consume its output without sharing
any of the method's code.
"""
from .synth import (  # noqa: F401
    Database,
    random_dag_database,
    subset_queries,
    random_queries,
    score_queries,
    zipf_item_probs,
    zipf_transaction_bitmaps,
    basket_transaction_bitmaps,
    weighted_itemsets,
    config_database,
    CONFIGS,
)
