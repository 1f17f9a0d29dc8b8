// Ensemble kernel instantiations for the collapsed volume rule.
#define ESDG_RULE 0
#include "esdg_ensemble_impl.cuh"
