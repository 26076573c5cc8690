// Persistent forest kernel for 2-dimensional points (see forest.cu).
#define FOREST_D 2
#include "forest_impl.cuh"
