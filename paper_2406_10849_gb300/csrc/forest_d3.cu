// Persistent forest kernel for 3-dimensional points (see forest.cu).
#define FOREST_D 3
#include "forest_impl.cuh"
