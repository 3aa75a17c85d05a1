"""GB300-native grid-hopping polygonizer (sm_103a CUDA behind a C ABI)."""
