"""The paper's value-count model -- TEST INFRASTRUCTURE ONLY.

Sec. III.B counts the metric values the approach computes for a system of
c classes and m methods: fan-in and fan-out once per method (2m), one
similarity value per unordered method pair (m(m-1)/2), and LCOM and CBO for
every class plus every class after receiving every method (c(m+1) each):

    #values = 2m + m(m-1)/2 + 2c(m+1)

Table I prints this count (in millions) for its 13 systems; the golden file
``tests/golden/table1_values.csv`` holds those printed rows.
"""


def count_values(c: int, m: int) -> int:
    fan = 2 * m
    similarity = m * (m - 1) // 2
    lcom_and_cbo = 2 * c * (m + 1)
    return fan + similarity + lcom_and_cbo


def lcom_values(c: int, m: int) -> int:
    """#LCOM values of Sec. III.B: each class, and each class after a move in."""
    return c + c * m
