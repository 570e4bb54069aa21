"""GB300-native SGD_Tucker: the minibatch SGD hot path of sparse Tucker
decomposition with a Kruskal-parameterised core (Li et al., arXiv 2012.03550),
as hand-written CUDA for sm_103a behind a small C ABI.

`binding` is the thin ctypes layer over libsgdtucker.so (same function names as
the C ABI); `synth` manufactures seeded synthetic inputs.
"""
__all__ = ["binding", "synth"]
