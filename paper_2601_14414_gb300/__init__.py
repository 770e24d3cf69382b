"""GB300-native (sm_103a) implementation of the piMPC hot path (arXiv 2601.14414)."""
