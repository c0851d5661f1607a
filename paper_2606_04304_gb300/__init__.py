"""GB300-native hot path of the OVRO-LWA ultra-narrowband all-sky imaging search.

``paper_2606_04304_gb300.ovro`` is the Python binding of the C-ABI library
``libovro.so`` (include/ovro.h); ``paper_2606_04304_gb300.build`` compiles it.
Importing the package itself loads nothing, so the build step can run without
a GPU.
"""
