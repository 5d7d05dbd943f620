"""CloakLM's cloaked linear layer, GB300-native (sm_103a).

``cloak`` binds the C ABI of libcloak (include/cloak.h); ``synth`` holds the
seeded synthetic shapes and inputs; ``build`` compiles the CUDA library.
The CUDA library is loaded on first use and its absence is an error.
"""
__all__ = ["cloak", "synth", "build"]
