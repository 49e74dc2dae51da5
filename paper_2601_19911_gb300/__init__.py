"""GB300-native key-only OLAP primitives: Top-K selection and hash-join
build/probe over (key, row-id) columns, and the Risky Gate cost estimator."""
