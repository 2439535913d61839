"""GB300-native depth stage of an active-stereo sensor simulator (arxiv 2201.11924, Sec. VI-D).

``simsense`` holds the Python binding of the CUDA library (``libsimsense.so``,
C ABI declared in ``include/simsense.h``); ``configs`` and ``scenes`` define
and synthesise the workloads.
"""
