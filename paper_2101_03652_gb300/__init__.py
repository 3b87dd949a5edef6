"""GB300-native single-source Personalized PageRank (PowerPush / SpeedPPR).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/ppr.h``); this package only marshals arguments to it.
"""
from .binding import (PPR_APPROX, PPR_FLAG_FIXED_PASSES, PPR_FLAG_FP32_ONLY, PPR_FLAG_INDEX, PPR_FLAG_NO_ACTIVE, PPR_FLAG_PARTIAL, PPR_FLAG_SYNC,
                      PPR_FLAG_TMA_GATHER, PPR_HP, Graph, Model, PPRError, load_library, ppr_default_opts, ppr_free,
                      ppr_graph_load, ppr_last_error, ppr_model_default_opts, ppr_sssp_query)

__all__ = ["Graph", "Model", "ppr_model_default_opts", "PPRError", "PPR_HP", "PPR_APPROX", "PPR_FLAG_PARTIAL",
           "PPR_FLAG_SYNC", "PPR_FLAG_INDEX", "PPR_FLAG_FIXED_PASSES", "PPR_FLAG_FP32_ONLY", "PPR_FLAG_NO_ACTIVE",
           "PPR_FLAG_TMA_GATHER", "load_library", "ppr_graph_load", "ppr_sssp_query",
           "ppr_free", "ppr_last_error", "ppr_default_opts"]
