// Collide kernel instantiations: float, 2D.
#define EF_T float
#define EF_D 2
#define EF_SUF f32_2d
#include "ef_collide_variant.inc"
