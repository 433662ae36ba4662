// Collide kernel instantiations: double, 2D.
#define EF_T double
#define EF_D 2
#define EF_SUF f64_2d
#include "ef_collide_variant.inc"
