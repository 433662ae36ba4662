// Collide kernel instantiations: float, 3D.
#define EF_T float
#define EF_D 3
#define EF_SUF f32_3d
#include "ef_collide_variant.inc"
