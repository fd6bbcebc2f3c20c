"""GB300-native budgeted group-by (hybrid-hash with Pre-Partitioning, plus a
radix-sort path), after Wen, Borkar, Carey and Tsotras, "Revisiting Aggregation
for Data Intensive Applications: A Performance Study".

The compute path is libagg.so (hand-written CUDA for sm_103a behind the C ABI
of include/agg.h); this package is its Python binding.
"""
from ._abi import (AGG_COUNT, AGG_I32, AGG_I64, AGG_MAX, AGG_MIN, AGG_PATH_AUTO, AGG_PATH_HASH, AGG_PATH_SORT,
                   AGG_SUM, AggError, agg_tuning)

__all__ = ["AGG_COUNT", "AGG_SUM", "AGG_MIN", "AGG_MAX", "AGG_I32", "AGG_I64", "AGG_PATH_HASH", "AGG_PATH_SORT",
           "AGG_PATH_AUTO", "AggError", "agg_tuning", "GroupBy"]


def __getattr__(name):
    if name == "GroupBy":
        from .groupby import GroupBy
        return GroupBy
    raise AttributeError(name)
