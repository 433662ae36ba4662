// Low-mode feature kernel instantiations: double.
#define EF_T double
#define EF_SUF f64
#include "ef_features_variant.inc"
