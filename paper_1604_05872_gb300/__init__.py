"""GB300-native batched element-local assembly (see include/fea.h)."""
