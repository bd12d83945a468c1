"""GB300-native (sm_103a) relational hot path: predicate filter with stream compaction, inner
hash join (build, probe) and hash group-by aggregation, behind the C-ABI library libsirius.so.

Importing the package loads nothing; ``paper_2508_04701_gb300.sirius`` loads the CUDA library
and raises if it has not been built.
"""
__version__ = "0.1.0"
