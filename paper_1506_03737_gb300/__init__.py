"""GB300-native COLA particle-mesh library (see include/colapm.h).

``paper_1506_03737_gb300.colapm`` is the ctypes binding of libcolapm.so, ``workloads`` the
named configurations and seeded synthetic inputs, ``build`` the in-tree nvcc build.
"""
