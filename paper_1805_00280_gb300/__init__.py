"""GB300-native node2vec 2nd-order walk sampler (Fast-Node2Vec hot path)."""
