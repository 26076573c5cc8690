// Persistent forest kernel for 1-dimensional points (see forest.cu).
#define FOREST_D 1
#include "forest_impl.cuh"
