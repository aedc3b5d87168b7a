"""GB300-native HashGraph (placeholder until the CUDA binding lands)."""
def load():
    raise RuntimeError("libhg.so not built yet")
