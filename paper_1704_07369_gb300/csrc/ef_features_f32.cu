// Low-mode feature kernel instantiations: float.
#define EF_T float
#define EF_SUF f32
#include "ef_features_variant.inc"
