// Batched LOBPCG for the filtered generalised eigenproblems of GenEO.
#include "setup.hpp"

namespace geneo {

void geneo_eigenvectors(geneo_ctx *c) {
  (void)c;
  throw Error(GENEO_ERR_INVALID_ARG, "GenEO eigensolver not built yet");
}

}  // namespace geneo
