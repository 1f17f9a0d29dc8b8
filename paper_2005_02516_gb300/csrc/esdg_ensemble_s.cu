// Ensemble kernel instantiations for the symmetric volume rule.
#define ESDG_RULE 1
#include "esdg_ensemble_impl.cuh"
