"""GB300-native forward-kinematics kernel proxy collision checking
(Das and Yip, arXiv 1910.06451).

``fkfast`` is the binding of the CUDA library libfkfast.so; ``synth`` draws
the seeded synthetic arms, obstacles and configurations; ``build`` compiles
the library for sm_103a.  Importing the package loads nothing: the library is
loaded by the first call into ``fkfast``.
"""
